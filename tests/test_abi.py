"""CPU-side checks of the C ABI: the library builds and loads without a GPU,
exports every function include/lbm_mix.h declares, and rejects bad
parameters before touching CUDA."""
import ctypes
import os
import re

import pytest

from paper_1603_08221_gb300 import binding
from paper_1603_08221_gb300 import build as cuda_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    cuda_build.build()
    return binding.load()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(lbm_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_header_declares_the_api():
    names = _declared()
    for n in ["lbm_mix_create", "lbm_mix_init", "lbm_mix_step", "lbm_mix_run_to_steady",
              "lbm_mix_moments", "lbm_mix_separation", "lbm_mix_destroy"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in sorted(_declared()):
        assert hasattr(lib, name), name
        assert name in binding._SIGS, f"binding lacks {name}"


def test_default_params(lib):
    p = binding.lbm_mix_default_params()
    assert p.m_a == 4.003 and p.m_b == 39.948 and p.C_l == 0.5
    assert p.tau_e == 1.1 and p.tau_eps == 1.2 and p.c_m0 == 1.016
    assert p.N == 16 and p.L_over_H == 20.0 and p.storage == binding.LBM_FP32
    # the last fields: a ctypes mirror out of step with the C struct fails here
    assert p.diag_every == 1 and p.reref_every == -1


@pytest.mark.parametrize("field,value", [
    ("C_l", 0.0), ("C_l", 1.0), ("theta", 0.5), ("Kn_out", 0.0), ("N", 1), ("m_a", -1.0),
    ("accommodation", 0.0), ("accommodation", 1.5), ("tau_e", 0.5), ("storage", 7),
    ("L_over_H", 0.1), ("x_periodic", 2), ("diag_every", 0), ("reref_every", -2),
])
def test_invalid_parameters_rejected_without_gpu(lib, field, value):
    p = binding.lbm_mix_default_params()
    setattr(p, field, value)
    h = ctypes.c_void_p()
    st = lib.lbm_mix_create(ctypes.byref(p), None, ctypes.byref(h))
    assert st == binding.LBM_EINVAL
    assert h.value is None
    assert binding.lbm_mix_last_error()


def test_null_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.lbm_mix_create(None, None, ctypes.byref(h)) == binding.LBM_EINVAL
    assert lib.lbm_mix_step(None, 1) == binding.LBM_EINVAL
    assert lib.lbm_mix_init(None) == binding.LBM_EINVAL
    assert lib.lbm_mix_launches_per_step(None) == binding.LBM_EINVAL
    assert lib.lbm_mix_tune_rows(None, None, 0, 10, None) == binding.LBM_EINVAL
    lib.lbm_mix_destroy(None)  # NULL-safe


def test_strerror(lib):
    for code in [0, -1, -2, -3, -4, -5, -6, -99]:
        assert binding.lbm_mix_strerror(code)


def test_too_large_lattice_rejected(lib):
    p = binding.lbm_mix_default_params()
    p.N = 8192
    p.N_x = 65536
    h = ctypes.c_void_p()
    assert lib.lbm_mix_create(ctypes.byref(p), None, ctypes.byref(h)) == binding.LBM_EINVAL


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(ImportError):
        binding._lib_backup = binding._lib
        try:
            binding._lib = None
            binding.load(str(tmp_path / "nope.so"))
        finally:
            binding._lib = binding._lib_backup


def test_sweep_rejects_bad_instances_without_gpu(lib):
    good = binding.lbm_mix_default_params()
    bad = binding.lbm_mix_default_params()
    bad.theta = 0.5
    low = binding.lbm_mix_default_params()
    low.storage = binding.LBM_BF16
    for plist in ([good, bad], [low]):
        arr = (binding.lbm_mix_params * len(plist))(*plist)
        s = ctypes.c_void_p()
        assert lib.lbm_sweep_create(arr, len(plist), ctypes.byref(s)) == binding.LBM_EINVAL
        assert s.value is None
    assert "instance 1" in binding.lbm_mix_last_error() or "FP32" in binding.lbm_mix_last_error()
    s = ctypes.c_void_p()
    assert lib.lbm_sweep_create(None, 0, ctypes.byref(s)) == binding.LBM_EINVAL


def test_adjoint_rejects_bad_arguments_without_gpu(lib):
    p = binding.lbm_mix_default_params()
    a = ctypes.c_void_p()
    for field, value in (("x_periodic", 1), ("theta", 0.5)):
        q = binding.lbm_mix_default_params()
        setattr(q, field, value)
        assert lib.lbm_adj_create(ctypes.byref(q), 100, 10, None, ctypes.byref(a)) == \
            binding.LBM_EINVAL
        assert a.value is None
    assert lib.lbm_adj_create(ctypes.byref(p), 0, 10, None, ctypes.byref(a)) == binding.LBM_EINVAL
    assert lib.lbm_adj_create(ctypes.byref(p), 100, 0, None, ctypes.byref(a)) == binding.LBM_EINVAL
