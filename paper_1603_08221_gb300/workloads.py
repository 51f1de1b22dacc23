"""Seeded synthetic workloads for the two-species microchannel problem.

This module holds problem definitions and random-number draws only: gas
pairs, the channel shapes of the paper's parametric study (Table 1 and the
20 x 700 lattice of Sec. 2) scaled to the benchmark sizes, random
post-collision states for the invariant tests and random wall accommodation
fields.  It contains none of the method's arithmetic, so both the CUDA path
and the FP64 oracle can take their inputs from it.
"""
from __future__ import annotations

import numpy as np

# Molecular masses (g/mol, standard atomic weights) of helium, neon and argon.
# The paper states only the mass ratios of its two mixtures, 1:10 for He-Ar
# and 1:2 for Ne-Ar (Sec. 2); these are the masses of the benchmark
# configurations, whose ratios round to those.
HE, NE, AR = 4.003, 20.18, 39.948

#: Named problems. Each is a dict of the physical inputs of Sec. 2 (masses,
#: light-species mole fraction, pressure ratio, outlet Knudsen number, cells
#: across the channel and aspect ratio).
PRESETS = {
    # He-Ar, 320 x 16 channel, 20 000 steps: GPU against the oracle.
    "heli_argon_320x16": dict(m_a=HE, m_b=AR, C_l=0.5, theta=2.0, Kn_out=0.1,
                              N=16, L_over_H=20.0),
    # Ne-Ar, 32768 x 512 channel: the throughput workload.
    "neon_argon_32768x512": dict(m_a=NE, m_b=AR, C_l=0.3, theta=3.0, Kn_out=0.05,
                                 N=512, L_over_H=64.0),
    # Its 1/16 linear-scale copy (2048 x 32), same C_l, theta, Kn_out.
    "neon_argon_2048x32": dict(m_a=NE, m_b=AR, C_l=0.3, theta=3.0, Kn_out=0.05,
                               N=32, L_over_H=64.0),
    # He-Ar 1280 x 64 (sensitivity workload shape).
    "heli_argon_1280x64": dict(m_a=HE, m_b=AR, C_l=0.5, theta=2.0, Kn_out=0.2,
                               N=64, L_over_H=20.0),
    # Ne-Ar 16384 x 256 (reduced-precision storage workload shape).
    "neon_argon_16384x256": dict(m_a=NE, m_b=AR, C_l=0.5, theta=2.5, Kn_out=0.5,
                                 N=256, L_over_H=64.0),
    # The paper's own lattice (20 x 700), Case 2 at Kn_out = 0.3, theta = 2.
    "paper_case2_700x20": dict(m_a=HE, m_b=AR, C_l=0.5, theta=2.0, Kn_out=0.3,
                               N=20, L_over_H=35.0),
}


def preset(name: str, **override) -> dict:
    p = dict(PRESETS[name])
    p.update(override)
    return p


def n_x(params: dict) -> int:
    """Number of lattice columns, N_x = round(N * L/H)."""
    if "N_x" in params:
        return int(params["N_x"])
    return int(round(params["N"] * params["L_over_H"]))


def random_post_state(N: int, N_x: int, seed: int, lo: float = 0.05,
                      hi: float = 0.15, dtype=np.float64) -> np.ndarray:
    """Non-negative random populations, layout [species][i][row][column].

    Species b gets ten times the mass of species a so that both carry
    comparable number densities for a 1:10 mass ratio."""
    rng = np.random.default_rng(seed)
    f = rng.uniform(lo, hi, size=(2, 9, N, N_x))
    f[1] *= 10.0
    return f.astype(dtype)


def random_accommodation(N_x: int, seed: int, spread: float = 0.05) -> np.ndarray:
    """Per-wall-node accommodation field, bottom wall then top wall, drawn as
    1 - U(0, spread) so that it stays in (0, 1]."""
    rng = np.random.default_rng(seed)
    return 1.0 - rng.uniform(0.0, spread, size=2 * N_x)


def sweep_instances(n: int = 96, seed: int = 0) -> list[dict]:
    """A parametric study in the spirit of Table 1 (gas pair, inlet
    composition, pressure ratio, Knudsen number, channel size), drawn with
    numpy's PCG64 from `seed`: He-Ar and Ne-Ar alternate, C_l cycles through
    0.1, 0.3, 0.5, 0.7, 0.9, theta ~ U[1.5, 5], Kn_out = 10^U[-2, 0],
    N from {16, 32, 64, 128} and L/H from {10, 20, 50}.  The draws are made
    in that order per instance."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(n):
        theta = float(rng.uniform(1.5, 5.0))
        kn = float(10.0 ** rng.uniform(-2.0, 0.0))
        N = int(rng.choice([16, 32, 64, 128]))
        LH = float(rng.choice([10.0, 20.0, 50.0]))
        out.append(dict(m_a=HE if k % 2 == 0 else NE, m_b=AR,
                        C_l=(0.1, 0.3, 0.5, 0.7, 0.9)[k % 5], theta=theta, Kn_out=kn,
                        N=N, L_over_H=LH))
    return out


def paper_table1(N: int = 20, L_over_H: float = 35.0) -> list[tuple[str, dict]]:
    """Every run of the paper's Table 1 on its 20 x 700 lattice: Cases 1-5
    He-Ar, 6-10 Ne-Ar, with (C_l,in, C_l,out, Kn_out, theta) as listed; the
    Kn_out and theta lists of Cases 2 and 7 are crossed."""
    rows = [
        (1, HE, 0.3, 0.3, (0.3,), (4.0,)),
        (2, HE, 0.5, 0.5, (0.3, 0.5, 1.0, 3.0, 5.0), (2.0, 3.0, 4.0, 5.0)),
        (3, HE, 0.7, 0.7, (0.3,), (4.0,)),
        (4, HE, 0.7, 0.3, (0.3, 1.0), (2.0,)),
        (5, HE, 0.3, 0.7, (0.3, 1.0), (2.0,)),
        (6, NE, 0.3, 0.3, (0.3,), (4.0,)),
        (7, NE, 0.5, 0.5, (0.3, 0.5, 1.0, 3.0, 5.0), (2.0, 3.0, 4.0, 5.0)),
        (8, NE, 0.7, 0.7, (0.3,), (4.0,)),
        (9, NE, 0.7, 0.3, (0.3, 1.0), (2.0,)),
        (10, NE, 0.3, 0.7, (0.3, 1.0), (2.0,)),
    ]
    out = []
    for case, m_a, cin, cout, kns, thetas in rows:
        for kn in kns:
            for th in thetas:
                out.append((f"case{case}_kn{kn:g}_theta{th:g}",
                            dict(m_a=m_a, m_b=AR, C_l=cin, C_l_out=cout, theta=th, Kn_out=kn,
                                 N=N, L_over_H=L_over_H)))
    return out
