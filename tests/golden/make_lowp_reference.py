"""Writes the FP64 oracle references of the 16-bit storage tests, computed by
the oracle alone, for copies of the Ne-Ar 16384 x 256 reduced-precision
workload (C_l = 0.5, theta = 2.5, Kn_out = 0.5, L/H = 64):

  lowp_neon_argon_2048x32.txt   the 1/8 linear-scale copy (N = 32) after
                                2000 and 20000 steps;
  lowp_neon_argon_1024x16.txt   the 1/16 copy (N = 16) at steady state
                                (STEADY_STEPS steps: its column-sum residual
                                over 1000 steps is below 1e-9 by then; at
                                1e-8, after 123 000 steps, CL still moves by
                                6 %).

The oracle takes about four hours of 8 cores to bring the 1/8 copy to
steady state, the 1/16 copy about an eighth of that, hence the two sizes.

Each file records, per horizon, the exact oracle's CL, C~_l, species mass
flows, light-species mole fraction C_l(x) at every NX/16-th column and the
species x velocities across the channel at columns N_x/4, N_x/2 and
3 N_x/4 ("exact" lines), and the error model of the storage: the same
quantities from the oracle with its post-collision deviations rounded every
step to BF16 or FP16 by stochastic rounding and re-referenced every 256
steps (as the library does), as differences from the exact run ("model"
lines; two generator seeds at 2000 steps, one otherwise).

Run: python tests/golden/make_lowp_reference.py short|steady"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
STEADY_STEPS = 206000
COLS_U = (0.25, 0.5, 0.75)
PARTS = {
    # name: (N, file, horizons, jobs (store_fmt, seed, horizons))
    "short": (32, "lowp_neon_argon_2048x32.txt", (2000, 20000),
              [(0, 0, (2000, 20000)), (2, 1, (2000, 20000)), (3, 1, (2000, 20000)),
               (2, 2, (2000,)), (3, 2, (2000,))]),
    "steady": (16, "lowp_neon_argon_1024x16.txt", (STEADY_STEPS,),
               [(0, 0, (STEADY_STEPS,)), (2, 1, (STEADY_STEPS,)), (3, 1, (STEADY_STEPS,))]),
}
NAMES = {2: "bf16_sr", 3: "fp16_sr"}


def params(N):
    sys.path.insert(0, ROOT)
    from paper_1603_08221_gb300 import workloads
    return dict(m_a=workloads.NE, m_b=workloads.AR, C_l=0.5, theta=2.5, Kn_out=0.5, N=N,
                L_over_H=64.0)


def observe(o):
    s = o.separation()
    m = o.moments()
    nx = o.N_x
    rec = {"CL": s["CL"], "Cl_tilde": s["Cl_tilde"], "mdot_a": s["mdot_a"],
           "mdot_b": s["mdot_b"], "Cl_profile": s["Cl_profile"][::nx // 16].copy()}
    for f in COLS_U:
        x = int(f * nx)
        rec[f"ua_x@{f}"] = m["ua_x"][:, x].copy()
        rec[f"ub_x@{f}"] = m["ub_x"][:, x].copy()
    return rec


def run(job):
    N, fmt, seed, horizons, threads = job
    os.environ["OMP_NUM_THREADS"] = str(threads)
    sys.path.insert(0, ROOT)
    import oracle
    p = params(N)
    if fmt:
        p.update(store_fmt=fmt, store_sr=1, reref_every=256, store_seed=seed)
    o = oracle.Oracle(p)
    o.init()
    out = {}
    for h in horizons:
        o.step(h - o.steps)
        out[h] = observe(o)
    return (fmt, seed), out


def fmt_vals(v):
    v = np.atleast_1d(np.asarray(v, dtype=float))
    return " ".join(f"{x:.17g}" for x in v)


def main(part):
    N, fname, horizons, jobs = PARTS[part]
    # the cores go to the long runs (the short ones finish early)
    longest = max(max(h) for _, _, h in jobs)
    n_long = sum(1 for _, _, h in jobs if max(h) == longest)
    spare = (os.cpu_count() or 1) - (len(jobs) - n_long)
    threads = {h: (max(1, spare // n_long) if max(h) == longest else 1) for _, _, h in jobs}
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        res = dict(pool.map(run, [(N, f, s, h, threads[h]) for f, s, h in jobs]))
    exact = res[(0, 0)]
    out = os.path.join(HERE, fname)
    with open(out, "w") as f:
        f.write(f"# FP64 oracle on the Ne-Ar {int(N * 64)} x {N} channel (C_l 0.5, theta 2.5, "
                "Kn_out 0.5); written by make_lowp_reference.py from oracle/ only.\n")
        f.write("# exact <steps> <key> <values...>: the exact oracle;\n")
        f.write("# model <storage> <seed> <steps> <key> <values...>: emulated storage minus exact\n")
        for h in horizons:
            for k, v in exact[h].items():
                f.write(f"exact {h} {k} {fmt_vals(v)}\n")
        for (fmt, seed), rec_h in sorted(res.items()):
            if fmt == 0:
                continue
            for h, rec in rec_h.items():
                for k, v in rec.items():
                    d = np.asarray(v, dtype=float) - np.asarray(exact[h][k], dtype=float)
                    f.write(f"model {NAMES[fmt]} {seed} {h} {k} {fmt_vals(d)}\n")
    print("wrote", out)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "short")
