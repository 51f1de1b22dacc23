"""FP64 CPU oracle for the two-species MRT lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use this package.  The CUDA library never
imports, links or falls back to it, and the two share no code.

The arithmetic lives in ``lbm_oracle.c`` (plain C, FP64, one OpenMP loop over
columns); this module compiles it with gcc and wraps it with ctypes.
``complex_step.py`` restates the same time integration in numpy on complex
numbers, for exact reference derivatives (complex step);
``reference_adjoint.py`` restates it with PyTorch CPU operations for a
reverse-mode reference gradient (torch.autograd).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``lbm_oracle.c`` into ``liblbm_oracle.so`` (gcc, -O2, OpenMP)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
           "-Wall", "-Wno-unused-function", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("m_a", ctypes.c_double), ("m_b", ctypes.c_double),
        ("C_l", ctypes.c_double), ("C_l_out", ctypes.c_double),
        ("theta", ctypes.c_double), ("Kn_out", ctypes.c_double),
        ("N", ctypes.c_int), ("N_x", ctypes.c_int),
        ("accommodation", ctypes.c_double), ("c_m0", ctypes.c_double),
        ("tau_rho", ctypes.c_double), ("tau_e", ctypes.c_double),
        ("tau_eps", ctypes.c_double),
        ("mu_ratio_a", ctypes.c_double), ("mu_ratio_b", ctypes.c_double),
        ("x_periodic", ctypes.c_int), ("y_periodic", ctypes.c_int),
        ("psi_off", ctypes.c_int), ("r_form", ctypes.c_int), ("lambda_pressure", ctypes.c_int),
        ("store_fmt", ctypes.c_int), ("store_sr", ctypes.c_int), ("reref_every", ctypes.c_int),
        ("store_seed", ctypes.c_uint), ("wall", ctypes.c_int),
    ]


_D = ctypes.c_double
_PD = ctypes.POINTER(ctypes.c_double)
_P = ctypes.c_void_p


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        sig = {
            "orc_E1": (_D, [_D]),
            "orc_psi": (_D, [_D]),
            "orc_dpsi": (_D, [_D]),
            "orc_Psi": (_D, [_D, _D, _D]),
            "orc_tau_q": (_D, [_D, _D, _D, _D]),
            "orc_tau_s_tilde": (_D, [_D, _D, _D, _D]),
            "orc_dbb_r": (_D, [_D, _D, _D]),
            "orc_feq": (None, [_D, _D, _D, _D, _PD]),
            "orc_matrix_M": (None, [_PD]),
            "orc_matrix_Minv": (None, [_PD]),
            "orc_create": (_P, [ctypes.POINTER(OrcParams)]),
            "orc_destroy": (None, [_P]),
            "orc_init": (None, [_P]),
            "orc_step": (None, [_P, ctypes.c_long]),
            "orc_set_post_state": (ctypes.c_int, [_P, _PD]),
            "orc_get_post_state": (None, [_P, _PD]),
            "orc_get_state": (None, [_P, _PD]),
            "orc_set_accommodation_field": (ctypes.c_int, [_P, _PD, ctypes.c_long]),
            "orc_moments": (None, [_P, _PD, _PD, _PD, _PD, _PD, _PD]),
            "orc_separation": (None, [_P, _PD, _PD, _PD, _PD, _PD,
                                      ctypes.POINTER(ctypes.c_int)]),
            "orc_face_flux": (None, [_P, _PD, _PD]),
            "orc_node_taus": (None, [_P, _PD, _PD, ctypes.c_int, _PD]),
            "orc_collide_node": (None, [_P, _PD, _PD, _PD, _PD, _PD]),
            "orc_constants": (None, [_P, _PD]),
            "orc_steps": (ctypes.c_long, [_P]),
            "orc_Nx": (ctypes.c_int, [_P]),
            "orc_num_threads": (ctypes.c_int, []),
            "orc_set_num_threads": (None, [ctypes.c_int]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_PD)


def E1(x: float) -> float:
    return _load().orc_E1(float(x))


def psi(a: float) -> float:
    return _load().orc_psi(float(a))


def dpsi(a: float) -> float:
    return _load().orc_dpsi(float(a))


def Psi(y: float, H: float, lam: float) -> float:
    return _load().orc_Psi(float(y), float(H), float(lam))


def tau_q(lam_w: float, mx_w: float, alpha: float, H: float) -> float:
    return _load().orc_tau_q(float(lam_w), float(mx_w), float(alpha), float(H))


def tau_s_tilde(y: float, H: float, lam: float, mx: float) -> float:
    return _load().orc_tau_s_tilde(float(y), float(H), float(lam), float(mx))


def dbb_r(c_m0: float, alpha: float, mx_w: float) -> float:
    return _load().orc_dbb_r(float(c_m0), float(alpha), float(mx_w))


def feq(rho_s: float, s_s: float, ux: float, uy: float) -> np.ndarray:
    out = np.zeros(9)
    _load().orc_feq(rho_s, s_s, ux, uy, _ptr(out))
    return out


def matrix_M() -> np.ndarray:
    out = np.zeros(81)
    _load().orc_matrix_M(_ptr(out))
    return out.reshape(9, 9)


def matrix_Minv() -> np.ndarray:
    out = np.zeros(81)
    _load().orc_matrix_Minv(_ptr(out))
    return out.reshape(9, 9)


def num_threads() -> int:
    return _load().orc_num_threads()


def set_num_threads(n: int) -> None:
    """Threads of the oracle's OpenMP loops; n < 1 restores the default."""
    _load().orc_set_num_threads(int(n))


_DEFAULTS = dict(C_l_out=-1.0, accommodation=1.0, c_m0=1.016, tau_rho=1.0,
                 tau_e=1.1, tau_eps=1.2, mu_ratio_a=1.0, mu_ratio_b=1.0,
                 x_periodic=0, y_periodic=0, psi_off=0, r_form=0, lambda_pressure=0,
                 store_fmt=0, store_sr=0, reref_every=0, store_seed=0, wall=0)


class Oracle:
    """One FP64 simulation.  ``params`` is a dict with the physical problem
    (m_a, m_b, C_l, theta, Kn_out, N, and either N_x or L_over_H) plus the
    optional knobs of ``_DEFAULTS``."""

    def __init__(self, params: dict):
        lib = _load()
        p = dict(_DEFAULTS)
        p.update({k: v for k, v in params.items()
                  if k in {f[0] for f in OrcParams._fields_} or k == "L_over_H"})
        if "N_x" not in p:
            p["N_x"] = int(round(p["N"] * p["L_over_H"]))
        p.pop("L_over_H", None)
        self.params = p
        self._p = OrcParams(**{f[0]: p[f[0]] for f in OrcParams._fields_})
        h = lib.orc_create(ctypes.byref(self._p))
        if not h:
            raise ValueError(f"oracle rejected parameters {p}")
        self._h = h
        self._lib = lib
        self.N = int(p["N"])
        self.N_x = int(p["N_x"])

    def close(self):
        if self._h:
            self._lib.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (2, 9, self.N, self.N_x)

    def init(self):
        self._lib.orc_init(self._h)

    def step(self, n: int = 1):
        self._lib.orc_step(self._h, int(n))

    @property
    def steps(self) -> int:
        return self._lib.orc_steps(self._h)

    def set_post_state(self, fp: np.ndarray):
        a = np.ascontiguousarray(fp, dtype=np.float64).reshape(self.shape)
        if self._lib.orc_set_post_state(self._h, _ptr(a)) != 0:
            raise ValueError("bad state")

    def get_post_state(self) -> np.ndarray:
        out = np.zeros(self.shape)
        self._lib.orc_get_post_state(self._h, _ptr(out))
        return out

    def get_state(self) -> np.ndarray:
        out = np.zeros(self.shape)
        self._lib.orc_get_state(self._h, _ptr(out))
        return out

    def set_accommodation_field(self, alpha: np.ndarray):
        a = np.ascontiguousarray(alpha, dtype=np.float64)
        if self._lib.orc_set_accommodation_field(self._h, _ptr(a), a.size) != 0:
            raise ValueError("bad accommodation field")

    def moments(self) -> dict:
        outs = [np.zeros((self.N, self.N_x)) for _ in range(6)]
        self._lib.orc_moments(self._h, *[_ptr(o) for o in outs])
        return dict(zip(["rho_a", "rho_b", "ua_x", "ua_y", "ub_x", "ub_y"], outs))

    def separation(self) -> dict:
        CL, Ct, ma, mb = (ctypes.c_double() for _ in range(4))
        xm = ctypes.c_int()
        prof = np.zeros(self.N_x)
        self._lib.orc_separation(self._h, ctypes.byref(CL), ctypes.byref(Ct),
                                 ctypes.byref(ma), ctypes.byref(mb), _ptr(prof),
                                 ctypes.byref(xm))
        return dict(CL=CL.value, Cl_tilde=Ct.value, mdot_a=ma.value,
                    mdot_b=mb.value, Cl_profile=prof, x_min=xm.value)

    def face_flux(self):
        Fa = np.zeros(self.N_x - 1)
        Fb = np.zeros(self.N_x - 1)
        self._lib.orc_face_flux(self._h, _ptr(Fa), _ptr(Fb))
        return Fa, Fb

    def node_taus(self, fa, fb, j: int) -> dict:
        fa = np.ascontiguousarray(fa, dtype=np.float64)
        fb = np.ascontiguousarray(fb, dtype=np.float64)
        out = np.zeros(8)
        self._lib.orc_node_taus(self._h, _ptr(fa), _ptr(fb), int(j), _ptr(out))
        return dict(zip(["tau_s", "tau_d", "lam", "lam_a", "lam_b", "mx", "ux", "uy"], out))

    def collide_node(self, fa, fb, tau):
        fa = np.ascontiguousarray(fa, dtype=np.float64)
        fb = np.ascontiguousarray(fb, dtype=np.float64)
        tau = np.ascontiguousarray(tau, dtype=np.float64)
        oa, ob = np.zeros(9), np.zeros(9)
        self._lib.orc_collide_node(self._h, _ptr(fa), _ptr(fb), _ptr(tau), _ptr(oa), _ptr(ob))
        return oa, ob

    def constants(self) -> dict:
        out = np.zeros(11)
        self._lib.orc_constants(self._h, _ptr(out))
        keys = ["mu", "mu_a", "mu_b", "rho_in_a", "rho_in_b", "rho_out_a",
                "rho_out_b", "s_a", "s_b", "mh_a", "mh_b"]
        return dict(zip(keys, out))
