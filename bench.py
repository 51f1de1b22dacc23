#!/usr/bin/env python3
"""Throughput benchmark of the fused two-species MRT-LBM step on GB300.

One benchmark step is one lattice Boltzmann time step of the whole hot path
(pull-stream + DBB walls + pressure ends + moments + effective relaxation
times + MRT collision + FP64 column reductions and separation diagnostics),
i.e. one launch of the fused kernel over the Ne-Ar 32768 x 512 channel
(16.8 M nodes, two species, 2.4 GB of FP32 populations: larger than L2, so no
flush is needed between steps).

Prints ONE JSON line (rank 0).  Beside the FP32 line it carries the BF16 /
FP16 storage timings, the 96-channel parametric sweep against sequential
lone runs, and the adjoint (gradient) time against the forward time.
--impl reference times the FP64 oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_NODE = 2 * 9 * 4 * 2  # two species x 9 populations x FP32 x (read + write)
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal (the roofline uses the measured copy rate)
WORKLOAD = "neon_argon_32768x512"
REF_SAMPLE = "neon_argon_2048x32"  # 1/16 linear-scale copy (same C_l, theta, Kn_out)
CPU_FULL_STEPS = 3  # oracle steps of the full workload timed for cpu_baseline
REF_MAX_STEPS = 20  # oracle steps of the full workload timed by --impl reference
KERNEL = "lbm_step_kernel"
TUNE_STEPS = 50  # timed steps per candidate schedule of lbm_mix_tune_rows
PROFILE_MD = os.path.join(ROOT, "profiles", "lbm_step_kernel_neon_argon_32768x512.md")
KERNEL_SRC = os.path.join(ROOT, "paper_1603_08221_gb300", "csrc", "lbm_mix.cu")
KERNEL_SECTION_END = b"// ------------------------------------------------------------ init kernels"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def aggregate(elapsed_per_rank, units_per_rank):
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    t = max(elapsed_per_rank)
    return sum(units_per_rank) / t, t


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(
                    ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                     "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                for line in out.stdout.strip().splitlines():
                    self.rows.append([c.strip() for c in line.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *exc):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) < 9:
                continue
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def profiled_traffic():
    """DRAM bytes per launch of the step kernel from the committed ncu
    summary, if it was taken on the current kernel source; else None."""
    try:
        text = open(PROFILE_MD).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    h = re.search(r"kernel_source_sha256:\s*([0-9a-f]+)", text)
    if not m or not h:
        return None
    return float(m.group(1)) if h.group(1) == kernel_source_sha256() else None


def kernel_source_sha256():
    """sha256 of the device-code part of the library source that the step
    kernel is built from (everything before the init kernels); host-side
    changes below that point leave the recorded counters valid."""
    text = open(KERNEL_SRC, "rb").read()
    end = text.find(KERNEL_SECTION_END)
    if end < 0:
        raise RuntimeError(f"marker {KERNEL_SECTION_END!r} missing from {KERNEL_SRC}")
    return hashlib.sha256(text[:end]).hexdigest()


def oracle_throughput(steps: int, sample: str, threads: int = 0, keep: bool = False):
    """FP64 oracle MLUPS on the host cores over `steps` steps of `sample`
    (threads >= 1: on that many OpenMP threads).  The timed steps follow one
    untimed step, so the oracle ends at step steps + 1; keep=True also
    returns it."""
    import oracle
    from paper_1603_08221_gb300 import workloads

    p = workloads.preset(sample)
    o = oracle.Oracle(p)
    oracle.set_num_threads(threads)
    try:
        o.init()
        o.step(1)  # untimed first step (page-in)
        t0 = time.perf_counter()
        o.step(steps)
        dt = time.perf_counter() - t0
        used = oracle.num_threads()
    finally:
        oracle.set_num_threads(0)
    nodes = o.N * (o.N_x - 2)
    out = (nodes * steps / dt / 1e6, dt, used, nodes)
    return out + (o,) if keep else out


def parity_against_oracle(o, stream):
    """Errors of the GPU FP32 path against the FP64 oracle object `o` after
    the same number of steps on the same channel: max |error| over the field
    relative to the field's max for rho_s, u_s (x and y, scaled by the
    largest |u_x|), and the scalar diagnostics."""
    import numpy as np
    from paper_1603_08221_gb300 import binding
    g = binding.LbmMix(stream=stream, **o.params_dict)
    g.init()
    g.step(o.steps)
    mg, mo = g.moments(), o.moments()
    sg, so = g.separation(), o.separation()
    g.close()
    uscale = max(np.abs(mo["ua_x"]).max(), np.abs(mo["ub_x"]).max())
    err = {"steps": o.steps,
           "rho_rel": max(float(np.abs(mg[k] - mo[k]).max() / np.abs(mo[k]).max())
                          for k in ("rho_a", "rho_b")),
           "u_rel": max(float(np.abs(mg[k] - mo[k]).max() / uscale)
                        for k in ("ua_x", "ua_y", "ub_x", "ub_y")),
           "CL": so["CL"], "CL_abs": abs(sg["CL"] - so["CL"]),
           "mdot_rel": max(abs(sg[k] - so[k]) / abs(so[k]) for k in ("mdot_a", "mdot_b")),
           "Cl_profile_abs": float(np.abs(sg["Cl_profile"] - so["Cl_profile"]).max())}
    return err


def run_sweep(args, rank, world, barrier):
    """The seeded 96-channel parametric study, every instance run to a
    steady-state residual of 1e-8 (or the step cap, or divergence), as one
    graph-replayed concurrent sweep with the schedule autotuner.  The
    sequential baseline (lone handles, plain launches, the same convergence
    test) is timed on every fourth instance and scaled to the whole study by
    node updates (each lone run takes exactly its instance's steps in the
    sweep).  Instances are dealt round-robin over the ranks."""
    from paper_1603_08221_gb300 import binding, workloads
    inst = workloads.sweep_instances()
    ids = [k for k in range(len(inst)) if k % world == rank]
    mine = [inst[k] for k in ids]
    tol, check = 1e-8, 1000
    sw = binding.LbmSweep(mine)
    sw.init()
    barrier()
    t0 = time.perf_counter()
    steps, _, status = sw.run_to_steady(tol, args.sweep_cap, check, autotune=True)
    barrier()
    t_sweep = time.perf_counter() - t0
    policy, _, round_ms = sw.schedule()
    sw.close()
    upd = [p["N"] * (workloads.n_x(p) - 2) * n for p, n in zip(mine, steps)]
    sub = [i for i, k in enumerate(ids) if k % args.sweep_seq_every == 0]
    t0 = time.perf_counter()
    for i in sub:
        g = binding.LbmMix(**mine[i])
        g.init()
        try:
            g.run_to_steady(tol, args.sweep_cap, check)
        except binding.LbmError as e:
            if e.status != binding.LBM_ENONFINITE:
                raise
        g.close()
    barrier()
    t_sub = time.perf_counter() - t0
    upd_sub = sum(upd[i] for i in sub)
    conv = [k for k, st in zip(ids, status) if st == binding.LBM_OK]
    capped = [k for k, st in zip(ids, status) if st == binding.LBM_ENOTCONVERGED]
    div = [k for k, st in zip(ids, status) if st == binding.LBM_ENONFINITE]
    updates = sum(upd)
    t_seq = t_sub * updates / max(upd_sub, 1)
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([t_sweep, t_seq, t_sub], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        c = torch.tensor([updates], dtype=torch.float64, device="cuda")
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
        t_sweep, t_seq, t_sub = float(t[0]), float(t[1]), float(t[2])
        updates = int(c[0])
        lists = [None] * world
        dist.all_gather_object(lists, (conv, capped, div))
        conv = sorted(k for l in lists for k in l[0])
        capped = sorted(k for l in lists for k in l[1])
        div = sorted(k for l in lists for k in l[2])
    return {"instances": len(inst), "tol": tol, "check_every": check,
            "step_cap": args.sweep_cap, "solves": len(conv), "seconds": t_sweep,
            "solves_per_s": len(conv) / t_sweep,
            "sequential_seconds": t_seq,
            "sequential_solves_per_s": len(conv) / t_seq, "speedup": t_seq / t_sweep,
            "sequential_sample": f"every {args.sweep_seq_every}th instance timed as lone runs "
                                 f"({t_sub:.1f} s), scaled by node updates",
            "aggregate_mlups": updates / t_sweep / 1e6,
            "outcomes": {"converged": len(conv), "step_cap": len(capped),
                         "diverged": len(div)},
            "diverged_instances": [dict(index=k, theta=round(inst[k]["theta"], 3),
                                        Kn_out=round(inst[k]["Kn_out"], 4), N=inst[k]["N"])
                                   for k in div],
            "capped_instances": capped,
            "autotuned_policy": policy, "autotune_block_ms": round_ms}


def run_adjoint(args, stream):
    """The sensitivity workload (He-Ar 1280 x 64, 5000 steps, accommodation
    1 - U(0, 0.05) per wall node): FP64 forward, one backward sweep for
    dCL/d(theta, Kn_out, alpha), and the FP32 forward of the same steps for
    the adjoint/forward time ratio.  The forward run keeps every step (one
    checkpoint interval: the backward sweep replays nothing) when that takes
    under half the free device memory; the same gradient with checkpoints
    every 70 steps (two replayed intervals in memory) is timed beside it."""
    import numpy as np
    import torch
    from paper_1603_08221_gb300 import binding, workloads
    p = workloads.preset("heli_argon_1280x64")
    nx = workloads.n_x(p)
    alpha = workloads.random_accommodation(nx, 1).reshape(2, nx)
    steps = args.adjoint_steps
    # per kept step: the state (18 N N_x), Psi values (6 N N_x), column data
    per_step = 8 * (24 * p["N"] * nx + 18 * nx + 4)
    free, _ = torch.cuda.mem_get_info()
    ck_lean = 70
    ck = steps if per_step * steps < 0.5 * free else ck_lean

    def timed(k):
        a = binding.LbmAdjoint(p, steps, k, alpha, stream=stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cl, _ = a.forward()
        t_f = time.perf_counter() - t0
        t0 = time.perf_counter()
        g = a.gradient(binding.LBM_ADJ_CL)
        t_g = time.perf_counter() - t0
        a.close()
        return cl, g, t_f, t_g

    cl, g, t_fwd64, t_grad = timed(ck)
    cl2, g2, t_fwd64_lean, t_grad_lean = timed(ck_lean)
    f = binding.LbmMix(stream=stream, **p)
    f.init()
    f.set_accommodation_field(np.ascontiguousarray(alpha.ravel()))
    f.step(10)
    f.sync()
    runs = []
    for _ in range(3):
        t0 = time.perf_counter()
        f.step(steps)
        f.sync()
        runs.append(time.perf_counter() - t0)
    t_fwd32 = sorted(runs)[1]
    return {"workload": "heli_argon_1280x64", "steps": steps, "checkpoint_every": ck,
            "kept_bytes": per_step * steps if ck == steps else None,
            "objective": "CL", "CL": cl, "dCL_dtheta": g["theta"], "dCL_dKn_out": g["Kn_out"],
            "dCL_dalpha_norm": float(np.linalg.norm(g["alpha"])),
            "forward_fp64_s": t_fwd64, "gradient_s": t_grad,
            "forward_fp32_s": t_fwd32, "forward_fp32_runs_s": runs,
            "adjoint_over_fp64_forward": t_grad / t_fwd64,
            "adjoint_over_fp32_forward": t_grad / t_fwd32,
            "forward_and_adjoint_over_fp32_forward": (t_fwd64 + t_grad) / t_fwd32,
            "checkpointed": {"checkpoint_every": ck_lean, "forward_fp64_s": t_fwd64_lean,
                             "gradient_s": t_grad_lean,
                             "adjoint_over_fp32_forward": t_grad_lean / t_fwd32,
                             "same_gradient": bool(g2["theta"] == g["theta"] and
                                                   g2["Kn_out"] == g["Kn_out"] and
                                                   np.array_equal(g2["alpha"], g["alpha"]))},
            "dtype": "f64 (forward, replay and adjoint)"}


def workload_config(name, p, N, N_x):
    """The config keys that name a workload (both arms report the same)."""
    return {"workload": name, "N": N, "N_x": N_x, "m_a": p["m_a"], "m_b": p["m_b"],
            "C_l": p["C_l"], "theta": p["theta"], "Kn_out": p["Kn_out"],
            "nodes_updated": N * (N_x - 2)}


def run_reference(args):
    """The oracle on the benchmark workload itself: min(K, REF_MAX_STEPS) full
    steps timed after min(W, 1) untimed ones, so that a run with a large K
    still ends within a few minutes."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    from paper_1603_08221_gb300 import workloads
    p = workloads.preset(args.workload)
    o = oracle.Oracle(p)
    o.init()
    o.step(min(args.warmup, 1))
    timed = max(1, min(args.steps, REF_MAX_STEPS))
    t0 = time.perf_counter()
    o.step(timed)
    dt = time.perf_counter() - t0
    nodes = o.N * (o.N_x - 2)
    mlups = nodes * timed / dt / 1e6
    sample = (f"FP64 oracle, {timed} steps of the {args.workload} workload itself "
              f"({nodes} nodes, {dt:.1f} s) after {min(args.warmup, 1)} untimed; "
              f"{args.steps} requested")
    line = {
        "impl": "reference", "metric": "MLUPS", "value": mlups, "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / timed * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.workload, p, o.N, o.N_x),
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1603_08221_gb300 import binding, workloads
    binding.load()
    storage = {"fp32": binding.LBM_FP32, "bf16": binding.LBM_BF16,
               "fp16": binding.LBM_FP16}[args.storage]
    p = workloads.preset(args.workload, diag_every=args.diag_every)
    # a dedicated (non-default) stream: the library and the CUDA events below
    # must see the same stream
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    sim = binding.LbmMix(stream=stream, storage=storage, **p)
    nodes = sim.N * (sim.N_x - 2)
    # schedule: rows per CTA timed over real steps (untimed setup), then the
    # run starts again from the initial state
    sim.init()
    if args.rows > 0:
        sim.set_rows_per_block(args.rows)
        rows = args.rows
    else:
        rows = sim.tune_rows(steps=TUNE_STEPS)
        sim.init()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    # ---------------- device-resident timing: K fused launches, inputs in HBM
    binding.lbm_mix_step(sim.h, args.warmup)
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        binding.lbm_mix_step(sim.h, args.steps)
        ev1.record(stream)
        ev1.synchronize()
    barrier()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    sep = sim.separation()  # raises on a non-finite state
    # kernels in the timed region: the step kernel, and the wall kernel ahead
    # of it where the library runs one (16-bit storage; FP32 grids of two or
    # more waves), per step; 16-bit storage adds, every 256 steps (counted
    # from the handle's first step), the two kernels of a re-reference
    per_step = binding.lbm_mix_launches_per_step(sim.h)
    # bytes of one population buffer (strips of 32 columns, 18 values per node)
    state_gb = 18 * sim.N * 32 * ((sim.N_x + 31) // 32) * (4 if args.storage == "fp32" else 2) / 1e9
    launches = args.steps * per_step
    if args.storage != "fp32":
        launches += 2 * ((args.warmup + args.steps) // 256 - args.warmup // 256)

    # ---------------- end to end through the C ABI with host buffers
    f_host = torch.empty((2, 9, sim.N, sim.N_x), dtype=torch.float32, pin_memory=True)
    f_np = f_host.numpy()
    f_np[...] = sim.get_post_state()
    outs = [torch.empty((sim.N, sim.N_x), dtype=torch.float64, pin_memory=True)
            for _ in range(6)]
    ptrs = [o.numpy() for o in outs]
    lib = binding.load()
    import ctypes
    barrier()
    t0 = time.perf_counter()
    binding.lbm_mix_set_post_state(sim.h, f_np)
    binding.lbm_mix_step(sim.h, args.steps)
    st = lib.lbm_mix_moments(sim.h, *[binding._dptr(a) for a in ptrs])
    assert st == 0, binding.lbm_mix_last_error()
    sep_e2e = sim.separation()
    barrier()
    e2e_elapsed = time.perf_counter() - t0
    h2d = f_np.nbytes
    d2h = sum(a.nbytes for a in ptrs) + 8 * (sim.N_x + 8)

    # ---------------- reduced-precision storage on the same workload (device timing)
    variants = {}
    if not args.no_variants:
        for name, storage in (("bf16", binding.LBM_BF16), ("fp16", binding.LBM_FP16)):
            v = binding.LbmMix(stream=stream, storage=storage, **p)
            v.init()
            if args.rows > 0:
                v.set_rows_per_block(args.rows)
                v_rows = args.rows
            else:
                v_rows = v.tune_rows(steps=TUNE_STEPS)
                v.init()
            binding.lbm_mix_step(v.h, args.warmup)
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            binding.lbm_mix_step(v.h, args.steps)
            e1.record(stream)
            e1.synchronize()
            t_v = e0.elapsed_time(e1) / 1e3 / args.steps
            variants[name] = {"ms_per_step": t_v * 1e3, "value": nodes / t_v / 1e6,
                              "unit": "MLUPS", "bytes_per_node_step": BYTES_PER_NODE // 2,
                              "achieved_gbs": BYTES_PER_NODE // 2 * nodes / t_v / 1e9,
                              "reref_every": 256, "rows_per_block": v_rows}
            del v

    sweep = None if args.no_sweep else run_sweep(args, rank, world, barrier)
    adjoint = None if (args.no_adjoint or rank != 0) else run_adjoint(args, stream)

    # ---------------- whole-job aggregation (max time over ranks)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([elapsed, e2e_elapsed], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed, e2e_elapsed = float(t[0]), float(t[1])
    mlups = aggregate([elapsed], [nodes * args.steps * world])[0] / 1e6
    e2e_mlups = nodes * args.steps * world / e2e_elapsed / 1e6
    ms_per_step = elapsed / args.steps * 1e3

    if rank != 0:
        return 0
    peak, peak_kind = measured_peak_hbm()
    bytes_per_node = BYTES_PER_NODE if args.storage == "fp32" else BYTES_PER_NODE // 2
    achieved = bytes_per_node * nodes / (elapsed / args.steps) / 1e9
    traffic = profiled_traffic() if args.storage == "fp32" else None
    cpu = None
    parity = None
    if world == 1 and not args.no_cpu_baseline:
        # all host cores on a bounded sample of the benchmark workload itself
        f_mlups, f_dt, cores, f_nodes = oracle_throughput(CPU_FULL_STEPS, args.workload)
        # the 1/16 linear-scale copy: the FP32 path's error after the same
        # steps (parity_vs_oracle) and the single-thread rate
        c_mlups, c_dt, _, c_nodes, o = oracle_throughput(args.cpu_steps - 1, REF_SAMPLE,
                                                         keep=True)
        s_steps = max(1, args.cpu_steps // 20)
        s_mlups, s_dt, _, _ = oracle_throughput(s_steps, REF_SAMPLE, threads=1)
        cpu = {"value": f_mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": f"FP64 oracle, {CPU_FULL_STEPS} steps of the {args.workload} "
                         f"workload itself ({f_nodes} nodes, {f_dt:.1f} s) after one untimed",
               "copy_1_16": {"value": c_mlups, "unit": "MLUPS", "cores": cores,
                             "sample": f"{args.cpu_steps} steps of the {REF_SAMPLE} 1/16 "
                                       f"linear-scale copy ({c_nodes} nodes, {c_dt:.1f} s)"},
               "single_thread": {"value": s_mlups, "unit": "MLUPS", "cores": 1,
                                 "sample": f"{s_steps} steps of the 1/16 copy ({s_dt:.1f} s)"}}
        o.params_dict = workloads.preset(REF_SAMPLE)
        parity = dict(workload=REF_SAMPLE, **parity_against_oracle(o, stream))
    line = {
        "metric": "MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": world,
        "value_per_species_set": 2 * mlups,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.storage == "fp32" else f"f32 compute, {args.storage} storage",
        "data": "synthetic",
        "config": {**workload_config(args.workload, p, sim.N, sim.N_x),
                   "bytes_per_node_step": bytes_per_node, "storage": args.storage,
                   "diag_every": args.diag_every,
                   "rows_per_block": rows,
                   "schedule": ("given (--rows)" if args.rows > 0 else
                                f"rows per CTA tuned over {TUNE_STEPS} steps per candidate "
                                "(lbm_mix_tune_rows) before init; not timed"),
                   "l2": (f"state (2 x {state_gb:.2f} GB {args.storage.upper()}) larger "
                          "than L2; no flush" if state_gb > 0.129 else
                          f"state (2 x {state_gb:.3f} GB) fits in L2: not a DRAM figure"),
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_source": peak_kind, "kernel": KERNEL,
                     "timed": ("whole step: the step kernel and the wall kernel ahead of it"
                               if per_step == 2 else "whole step: the step kernel"),
                     "nominal_peak": NOMINAL_HBM_GBS,
                     "frac_of_nominal": achieved / NOMINAL_HBM_GBS},
        "cpu_baseline": cpu,
        "parity_vs_oracle": parity,
        "e2e": {"value": e2e_mlups, "unit": "MLUPS", "h2d_bytes_per_step": h2d / args.steps,
                "d2h_bytes_per_step": d2h / args.steps},
        "gpu_launches": launches,
        "storage_variants": variants or None,
        "sweep": sweep,
        "adjoint": adjoint,
        "clocks": clk.summary(),
        "result": {"CL": sep["CL"], "Cl_tilde": sep["Cl_tilde"], "mdot_a": sep["mdot_a"],
                   "mdot_b": sep["mdot_b"], "CL_e2e_run": sep_e2e["CL"]},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--rows", type=int, default=0,
                    help="rows per CTA of the step kernel; 0 = tune (lbm_mix_tune_rows)")
    ap.add_argument("--storage", choices=["fp32", "bf16", "fp16"], default="fp32",
                    help="population storage of the timed channel (FP32 is the headline)")
    ap.add_argument("--cpu-steps", type=int, default=2000,
                    help="oracle steps of the 1/16 copy: the CPU baseline and the parity check")
    ap.add_argument("--diag-every", type=int, default=100,
                    help="steps between FP64 separation-diagnostic reductions (the column "
                         "sums of the end columns are reduced every step)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the BF16/FP16 storage timings")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the adjoint (gradient) timing")
    ap.add_argument("--adjoint-steps", type=int, default=5000,
                    help="steps of the adjoint workload (5000 for the sensitivity study)")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the 96-channel parametric sweep")
    ap.add_argument("--sweep-cap", type=int, default=200000,
                    help="step cap per sweep instance")
    ap.add_argument("--sweep-seq-every", type=int, default=4,
                    help="time every n-th sweep instance as a lone run for the sequential "
                         "baseline")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
