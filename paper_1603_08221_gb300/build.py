"""Compiles the CUDA library ``liblbm_mix.so`` in-tree for sm_103a with nvcc."""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc", "lbm_mix.cu")
SRCS = [SRC, os.path.join(HERE, "csrc", "lbm_adjoint.cu")]
HDR = os.path.join(ROOT, "include", "lbm_mix.h")
INTERNAL_HDR = os.path.join(HERE, "csrc", "lbm_internal.h")
LIB = os.path.join(HERE, "liblbm_mix.so")

NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo",
              "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def build(force: bool = False, verbose: bool = False) -> str:
    """Builds liblbm_mix.so unless it is newer than its sources: each
    translation unit is compiled in parallel, then linked."""
    deps = SRCS + [HDR, INTERNAL_HDR]
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(s) for s in deps)):
        return LIB
    tag = f".tmp{os.getpid()}"
    objs = [os.path.splitext(s)[0] + tag + ".o" for s in SRCS]
    procs = [subprocess.Popen([nvcc(), *NVCC_FLAGS, "-c", src, "-o", obj],
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
             for src, obj in zip(SRCS, objs)]
    logs = []
    failed = False
    for pr in procs:
        out, err = pr.communicate()
        logs.append(err)
        failed |= pr.returncode != 0
    try:
        if failed:
            raise RuntimeError("nvcc failed:\n" + "\n".join(logs))
        tmp = LIB + tag
        res = subprocess.run([nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-shared",
                              *objs, "-o", tmp], capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed ({res.returncode}):\n{res.stdout}\n{res.stderr}")
        if verbose:
            print("\n".join(logs))
        os.replace(tmp, LIB)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return LIB
