"""ctypes binding of the C ABI declared in include/lbm_mix.h.

Argument marshalling only: every function here forwards to the function of
the same name in ``liblbm_mix.so`` (sm_103a CUDA).  There is no CPU path; if
the library has not been built, loading raises.  Streams may be given as
integers (``torch.cuda.Stream.cuda_stream``) or objects with a
``cuda_stream`` attribute.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm_mix.so")

LBM_OK = 0
LBM_EINVAL = -1
LBM_ENOMEM = -2
LBM_ECUDA = -3
LBM_ENONFINITE = -4
LBM_ENOTCONVERGED = -5
LBM_ETIMEOUT = -6
LBM_FP32 = 0
LBM_BF16 = 1
LBM_FP16 = 2
LBM_ROUND_STOCHASTIC = 0
LBM_ROUND_NEAREST = 1
LBM_WALL_DBB = 0
LBM_WALL_BSR = 1
LBM_R_FIRST = 0
LBM_R_SPECIES = 1
LBM_R_SECOND = 2


class lbm_mix_params(ctypes.Structure):
    _fields_ = [
        ("m_a", ctypes.c_double), ("m_b", ctypes.c_double),
        ("C_l", ctypes.c_double), ("C_l_out", ctypes.c_double),
        ("theta", ctypes.c_double), ("Kn_out", ctypes.c_double),
        ("N", ctypes.c_int), ("N_x", ctypes.c_int),
        ("L_over_H", ctypes.c_double),
        ("accommodation", ctypes.c_double), ("c_m0", ctypes.c_double),
        ("tau_rho", ctypes.c_double), ("tau_e", ctypes.c_double),
        ("tau_eps", ctypes.c_double),
        ("mu_ratio_a", ctypes.c_double), ("mu_ratio_b", ctypes.c_double),
        ("storage", ctypes.c_int), ("x_periodic", ctypes.c_int),
        ("diag_every", ctypes.c_int),
        ("reref_every", ctypes.c_int),
        ("rounding", ctypes.c_int),
        ("wall", ctypes.c_int),
        ("r_form", ctypes.c_int), ("lambda_pressure", ctypes.c_int),
    ]


class LbmError(RuntimeError):
    def __init__(self, status: int, func: str, message: str):
        super().__init__(f"{func}: {message} (status {status})")
        self.status = status


_D = ctypes.c_double
_PD = ctypes.POINTER(ctypes.c_double)
_PF = ctypes.POINTER(ctypes.c_float)
_H = ctypes.c_void_p
_I = ctypes.c_int
_L = ctypes.c_long

_SIGS = {
    "lbm_mix_default_params": (None, [ctypes.POINTER(lbm_mix_params)]),
    "lbm_mix_create": (_I, [ctypes.POINTER(lbm_mix_params), ctypes.c_void_p,
                            ctypes.POINTER(ctypes.c_void_p)]),
    "lbm_mix_destroy": (None, [_H]),
    "lbm_mix_init": (_I, [_H]),
    "lbm_mix_step": (_I, [_H, _L]),
    "lbm_mix_rereference": (_I, [_H]),
    "lbm_mix_run_to_steady": (_I, [_H, _D, _L, _L, ctypes.POINTER(_L), _PD]),
    "lbm_mix_moments": (_I, [_H, _PD, _PD, _PD, _PD, _PD, _PD]),
    "lbm_mix_moments_device": (_I, [_H, ctypes.c_void_p]),
    "lbm_mix_separation": (_I, [_H, _PD, _PD, _PD, _PD, _PD, ctypes.POINTER(_I)]),
    "lbm_mix_history": (_I, [_H, _PD, _L, ctypes.POINTER(_L)]),
    "lbm_mix_volume_flow": (_I, [_H, _I, _PD]),
    "lbm_mix_device_ptrs": (_I, [_H, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(_L),
                                 ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                 ctypes.POINTER(ctypes.c_void_p)]),
    "lbm_mix_set_accommodation_field": (_I, [_H, _PD, _L]),
    "lbm_mix_set_post_state": (_I, [_H, _PF, _L]),
    "lbm_mix_get_post_state": (_I, [_H, _PF, _L]),
    "lbm_mix_get_post_state_f64": (_I, [_H, _PD, _L]),
    "lbm_mix_dims": (_I, [_H, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_L)]),
    "lbm_mix_launches_per_step": (_I, [_H]),
    "lbm_mix_sync": (_I, [_H]),
    "lbm_mix_eval_special": (_I, [_PD, _PD, _PD, _L]),
    "lbm_mix_step_noalloc": (_I, [ctypes.POINTER(lbm_mix_params)] + [ctypes.c_void_p] * 9),
    "lbm_mix_set_rows_per_block": (_I, [_H, _I]),
    "lbm_mix_tune_rows": (_I, [_H, ctypes.POINTER(_I), _I, _L, ctypes.POINTER(_I)]),
    "lbm_sweep_create": (_I, [ctypes.POINTER(lbm_mix_params), _I,
                              ctypes.POINTER(ctypes.c_void_p)]),
    "lbm_sweep_destroy": (None, [_H]),
    "lbm_sweep_init": (_I, [_H]),
    "lbm_sweep_step": (_I, [_H, _L]),
    "lbm_sweep_run_to_steady": (_I, [_H, _D, _L, _L, _I, ctypes.POINTER(_L), _PD,
                                     ctypes.POINTER(_I)]),
    "lbm_sweep_instance": (_I, [_H, _I, ctypes.POINTER(ctypes.c_void_p)]),
    "lbm_sweep_schedule": (_I, [_H, ctypes.POINTER(_I), ctypes.POINTER(_I), _PD]),
    "lbm_adj_create": (_I, [ctypes.POINTER(lbm_mix_params), _L, _I, ctypes.c_void_p,
                            ctypes.POINTER(ctypes.c_void_p)]),
    "lbm_adj_destroy": (None, [_H]),
    "lbm_adj_set_accommodation_field": (_I, [_H, _PD, _L]),
    "lbm_adj_forward": (_I, [_H, _PD, _PD]),
    "lbm_adj_state": (_I, [_H, _PD, _L]),
    "lbm_adj_gradient": (_I, [_H, _I, _PD, _PD, _PD, _L]),
    "lbm_mix_strerror": (ctypes.c_char_p, [_I]),
    "lbm_mix_last_error": (ctypes.c_char_p, []),
}

_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads liblbm_mix.so; raises if it is missing (no fallback exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError(
                f"{path} is missing: build the CUDA library first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(status: int, func: str):
    if status != LBM_OK:
        msg = _lib.lbm_mix_last_error().decode() or _lib.lbm_mix_strerror(status).decode()
        raise LbmError(status, func, msg)


def _dptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_PD)


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return int(stream.cuda_stream)
    return int(stream)


# ------------------------------------------------ same-name thin wrappers
def lbm_mix_default_params() -> lbm_mix_params:
    p = lbm_mix_params()
    load().lbm_mix_default_params(ctypes.byref(p))
    return p


def lbm_mix_create(params: lbm_mix_params, stream=None) -> int:
    lib = load()
    h = ctypes.c_void_p()
    _check(lib.lbm_mix_create(ctypes.byref(params), _stream_handle(stream), ctypes.byref(h)),
           "lbm_mix_create")
    return h.value


def lbm_mix_destroy(h) -> None:
    load().lbm_mix_destroy(h)


def lbm_mix_init(h) -> None:
    _check(load().lbm_mix_init(h), "lbm_mix_init")


def lbm_mix_step(h, nsteps: int) -> None:
    _check(load().lbm_mix_step(h, int(nsteps)), "lbm_mix_step")


def lbm_mix_rereference(h) -> None:
    _check(load().lbm_mix_rereference(h), "lbm_mix_rereference")


def lbm_mix_run_to_steady(h, tol: float, max_steps: int, check_every: int):
    steps = _L()
    res = _D()
    st = load().lbm_mix_run_to_steady(h, float(tol), int(max_steps), int(check_every),
                                      ctypes.byref(steps), ctypes.byref(res))
    if st not in (LBM_OK, LBM_ENOTCONVERGED):
        _check(st, "lbm_mix_run_to_steady")
    return st, steps.value, res.value


def lbm_mix_dims(h):
    N, Nx, steps = _I(), _I(), _L()
    _check(load().lbm_mix_dims(h, ctypes.byref(N), ctypes.byref(Nx), ctypes.byref(steps)),
           "lbm_mix_dims")
    return N.value, Nx.value, steps.value


def lbm_mix_launches_per_step(h) -> int:
    n = load().lbm_mix_launches_per_step(h)
    if n < 0:
        _check(n, "lbm_mix_launches_per_step")
    return n


def lbm_mix_moments(h) -> dict:
    N, Nx, _ = lbm_mix_dims(h)
    outs = [np.empty((N, Nx)) for _ in range(6)]
    _check(load().lbm_mix_moments(h, *[_dptr(o) for o in outs]), "lbm_mix_moments")
    return dict(zip(["rho_a", "rho_b", "ua_x", "ua_y", "ub_x", "ub_y"], outs))


def lbm_mix_moments_device(h, d_out_ptr: int) -> None:
    _check(load().lbm_mix_moments_device(h, ctypes.c_void_p(int(d_out_ptr))),
           "lbm_mix_moments_device")


def lbm_mix_device_ptrs(h) -> dict:
    pop, refrho, alpha, cs = (ctypes.c_void_p() for _ in range(4))
    n = _L()
    _check(load().lbm_mix_device_ptrs(h, ctypes.byref(pop), ctypes.byref(n), ctypes.byref(refrho),
                                      ctypes.byref(alpha), ctypes.byref(cs)),
           "lbm_mix_device_ptrs")
    return {"populations": pop.value, "n_populations": n.value, "refrho": refrho.value,
            "alpha": alpha.value, "colsum": cs.value}


class _DeviceArray:
    """A CUDA array interface (version 3) over library-owned device memory,
    so that torch.as_tensor (or any consumer of the interface) views it
    without a copy."""

    def __init__(self, ptr: int, shape: tuple, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3,
                                         "strides": None}


def lbm_mix_volume_flow(h, x: int = -1) -> float:
    q = _D()
    _check(load().lbm_mix_volume_flow(h, int(x), ctypes.byref(q)), "lbm_mix_volume_flow")
    return q.value


def lbm_mix_separation(h) -> dict:
    _, Nx, _ = lbm_mix_dims(h)
    CL, Ct, ma, mb = _D(), _D(), _D(), _D()
    xm = _I()
    prof = np.empty(Nx)
    _check(load().lbm_mix_separation(h, ctypes.byref(CL), ctypes.byref(Ct), ctypes.byref(ma),
                                     ctypes.byref(mb), _dptr(prof), ctypes.byref(xm)),
           "lbm_mix_separation")
    return dict(CL=CL.value, Cl_tilde=Ct.value, mdot_a=ma.value, mdot_b=mb.value,
                Cl_profile=prof, x_min=xm.value)


def lbm_mix_history(h, max_records: int = 4096) -> np.ndarray:
    rec = np.zeros((max_records, 8))
    cnt = _L()
    _check(load().lbm_mix_history(h, _dptr(rec), int(max_records), ctypes.byref(cnt)),
           "lbm_mix_history")
    return rec[:cnt.value]


def lbm_mix_set_accommodation_field(h, alpha: np.ndarray) -> None:
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    _check(load().lbm_mix_set_accommodation_field(h, _dptr(a), a.size),
           "lbm_mix_set_accommodation_field")


def lbm_mix_set_post_state(h, f: np.ndarray) -> None:
    a = np.ascontiguousarray(f, dtype=np.float32)
    _check(load().lbm_mix_set_post_state(h, a.ctypes.data_as(_PF), a.size),
           "lbm_mix_set_post_state")


def lbm_mix_get_post_state(h) -> np.ndarray:
    N, Nx, _ = lbm_mix_dims(h)
    out = np.empty((2, 9, N, Nx), dtype=np.float32)
    _check(load().lbm_mix_get_post_state(h, out.ctypes.data_as(_PF), out.size),
           "lbm_mix_get_post_state")
    return out


def lbm_mix_get_post_state_f64(h) -> np.ndarray:
    N, Nx, _ = lbm_mix_dims(h)
    out = np.empty((2, 9, N, Nx), dtype=np.float64)
    _check(load().lbm_mix_get_post_state_f64(h, _dptr(out), out.size),
           "lbm_mix_get_post_state_f64")
    return out


def lbm_mix_sync(h) -> None:
    _check(load().lbm_mix_sync(h), "lbm_mix_sync")


def lbm_mix_eval_special(x: np.ndarray):
    x = np.ascontiguousarray(x, dtype=np.float64)
    e1 = np.empty_like(x)
    ps = np.empty_like(x)
    _check(load().lbm_mix_eval_special(_dptr(x), _dptr(e1), _dptr(ps), x.size),
           "lbm_mix_eval_special")
    return e1, ps


def lbm_mix_step_noalloc(params: lbm_mix_params, d_in: int, d_out: int, d_refrho: int,
                         d_alpha: int, d_colsum_in: int, d_colsum_out: int, d_record: int,
                         d_cl_profile: int, stream=None) -> None:
    """One allocation-free step on caller-owned device buffers (integer
    device addresses, e.g. torch ``data_ptr()``); see include/lbm_mix.h."""
    ptrs = [d_in, d_out, d_refrho, d_alpha, d_colsum_in, d_colsum_out, d_record, d_cl_profile]
    _check(load().lbm_mix_step_noalloc(ctypes.byref(params),
                                       *[ctypes.c_void_p(int(q)) for q in ptrs],
                                       ctypes.c_void_p(_stream_handle(stream))),
           "lbm_mix_step_noalloc")


def lbm_mix_strerror(status: int) -> str:
    return load().lbm_mix_strerror(int(status)).decode()


def lbm_mix_last_error() -> str:
    return load().lbm_mix_last_error().decode()


# --------------------------------------------------------- convenience
def make_params(**kw) -> lbm_mix_params:
    """Default parameters updated from keyword arguments (names of the C
    struct; ``L_over_H`` or ``N_x`` select the length)."""
    p = lbm_mix_default_params()
    names = {f[0] for f in lbm_mix_params._fields_}
    for k, v in kw.items():
        if k not in names:
            raise KeyError(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


def lbm_mix_set_rows_per_block(h, rows: int) -> None:
    _check(load().lbm_mix_set_rows_per_block(h, int(rows)), "lbm_mix_set_rows_per_block")


def lbm_mix_tune_rows(h, candidates=None, steps: int = 20) -> int:
    """Times `steps` real steps under each candidate rows-per-CTA (None: the
    library's list) and keeps the fastest; returns it.  Advances the state."""
    best = _I()
    if candidates is None:
        arr, n = None, 0
    else:
        arr = (_I * len(candidates))(*[int(c) for c in candidates])
        n = len(candidates)
    _check(load().lbm_mix_tune_rows(h, arr, n, int(steps), ctypes.byref(best)),
           "lbm_mix_tune_rows")
    return best.value


LBM_SWEEP_NPOLICY = 5


def lbm_sweep_create(params_list) -> ctypes.c_void_p:
    arr = (lbm_mix_params * len(params_list))(*params_list)
    h = ctypes.c_void_p()
    _check(load().lbm_sweep_create(arr, len(params_list), ctypes.byref(h)), "lbm_sweep_create")
    return h


def lbm_sweep_destroy(s) -> None:
    load().lbm_sweep_destroy(s)


def lbm_sweep_init(s) -> None:
    _check(load().lbm_sweep_init(s), "lbm_sweep_init")


def lbm_sweep_step(s, nsteps: int) -> None:
    _check(load().lbm_sweep_step(s, int(nsteps)), "lbm_sweep_step")


def lbm_sweep_run_to_steady(s, n: int, tol: float, max_steps: int, check_every: int,
                            autotune: bool):
    steps = (_L * n)()
    res = (_D * n)()
    status = (_I * n)()
    _check(load().lbm_sweep_run_to_steady(s, float(tol), int(max_steps), int(check_every),
                                          1 if autotune else 0, steps, res, status),
           "lbm_sweep_run_to_steady")
    return list(steps), list(res), list(status)


def lbm_sweep_instance(s, k: int) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load().lbm_sweep_instance(s, int(k), ctypes.byref(h)), "lbm_sweep_instance")
    return h


def lbm_sweep_schedule(s, n: int):
    pol = _I()
    rows = (_I * n)()
    ms = (_D * LBM_SWEEP_NPOLICY)()
    _check(load().lbm_sweep_schedule(s, ctypes.byref(pol), rows, ms), "lbm_sweep_schedule")
    return pol.value, list(rows), list(ms)


class LbmMix:
    """Owns one handle; methods forward to the same-name C functions."""

    def __init__(self, stream=None, **params):
        self.params = make_params(**params)
        self.h = lbm_mix_create(self.params, stream)
        self._owned = True
        self.N, self.N_x, _ = lbm_mix_dims(self.h)

    @classmethod
    def borrowed(cls, h, params: lbm_mix_params):
        """A view of a handle owned elsewhere (a sweep instance); never
        destroys it."""
        self = cls.__new__(cls)
        self.params = params
        self.h = h
        self._owned = False
        self.N, self.N_x, _ = lbm_mix_dims(self.h)
        return self

    def close(self):
        if getattr(self, "h", None):
            if getattr(self, "_owned", True):
                lbm_mix_destroy(self.h)
            self.h = None

    def set_rows_per_block(self, rows: int):
        lbm_mix_set_rows_per_block(self.h, rows)

    def tune_rows(self, candidates=None, steps: int = 20) -> int:
        return lbm_mix_tune_rows(self.h, candidates, steps)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def init(self):
        lbm_mix_init(self.h)

    def step(self, n: int = 1):
        lbm_mix_step(self.h, n)

    def rereference(self):
        lbm_mix_rereference(self.h)

    def sync(self):
        lbm_mix_sync(self.h)

    @property
    def steps(self) -> int:
        return lbm_mix_dims(self.h)[2]

    def moments(self) -> dict:
        return lbm_mix_moments(self.h)

    def separation(self) -> dict:
        return lbm_mix_separation(self.h)

    def volume_flow(self, x: int = -1) -> float:
        return lbm_mix_volume_flow(self.h, x)

    def device_views(self) -> dict:
        """Zero-copy CUDA array interfaces of the current state (valid until
        the next step): populations (stored deviations, strip layout, storage
        type), refrho and alpha (float [2][N_x]) and the column sums (FP64
        [4][N_x]).  Pass each to torch.as_tensor(..., device='cuda').  BF16
        populations appear as raw 16-bit words (the interface has no
        bfloat16 type): view them with .view(torch.bfloat16)."""
        d = lbm_mix_device_ptrs(self.h)
        st = self.params.storage
        typestr = "<f4" if st == LBM_FP32 else "<f2" if st == LBM_FP16 else "<u2"
        return {"populations": _DeviceArray(d["populations"], (d["n_populations"],), typestr),
                "refrho": _DeviceArray(d["refrho"], (2, self.N_x), "<f4"),
                "alpha": _DeviceArray(d["alpha"], (2, self.N_x), "<f4"),
                "colsum": _DeviceArray(d["colsum"], (4, self.N_x), "<f8")}

    def history(self, max_records: int = 4096) -> np.ndarray:
        return lbm_mix_history(self.h, max_records)

    def set_accommodation_field(self, alpha):
        lbm_mix_set_accommodation_field(self.h, alpha)

    def set_post_state(self, f):
        lbm_mix_set_post_state(self.h, f)

    def get_post_state(self) -> np.ndarray:
        return lbm_mix_get_post_state(self.h)

    def get_post_state_f64(self) -> np.ndarray:
        return lbm_mix_get_post_state_f64(self.h)

    def run_to_steady(self, tol: float, max_steps: int, check_every: int = 100):
        return lbm_mix_run_to_steady(self.h, tol, max_steps, check_every)


class LbmSweep:
    """Owns a sweep of independent channels (one parameter dict each)."""

    def __init__(self, params_list):
        self.params = [make_params(**p) for p in params_list]
        self.n = len(self.params)
        self.s = lbm_sweep_create(self.params)
        self._views = [None] * self.n

    def close(self):
        if getattr(self, "s", None):
            self._views = []
            lbm_sweep_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self):
        lbm_sweep_init(self.s)

    def step(self, n: int):
        lbm_sweep_step(self.s, n)

    def run_to_steady(self, tol: float, max_steps: int, check_every: int = 1000,
                      autotune: bool = False):
        """Per-instance (steps, residual, status) lists."""
        return lbm_sweep_run_to_steady(self.s, self.n, tol, max_steps, check_every, autotune)

    def instance(self, k: int) -> LbmMix:
        if self._views[k] is None:
            self._views[k] = LbmMix.borrowed(lbm_sweep_instance(self.s, k), self.params[k])
        return self._views[k]

    def schedule(self):
        """(policy, rows per CTA of each instance, autotuner block times in ms)."""
        return lbm_sweep_schedule(self.s, self.n)


LBM_ADJ_CL = 0
LBM_ADJ_FLUX = 1


class LbmAdjoint:
    """FP64 forward run of nsteps steps with checkpoints and its discrete
    adjoint (lbm_adj_* of the C ABI).  ``alpha``: optional [2][N_x]
    accommodation field (bottom wall, then top)."""

    def __init__(self, params: dict, nsteps: int, checkpoint_every: int = 70, alpha=None,
                 stream=None):
        self.params = make_params(**params)
        lib = load()
        h = ctypes.c_void_p()
        st = lib.lbm_adj_create(ctypes.byref(self.params), int(nsteps), int(checkpoint_every),
                                _stream_handle(stream), ctypes.byref(h))
        _check(st, "lbm_adj_create")
        self.h = h
        self.N = self.params.N
        self.N_x = self.params.N_x if self.params.N_x > 0 else int(
            round(self.params.N * self.params.L_over_H))
        if alpha is not None:
            a = np.ascontiguousarray(np.asarray(alpha, dtype=np.float64).ravel())
            _check(lib.lbm_adj_set_accommodation_field(self.h, _dptr(a), a.size),
                   "lbm_adj_set_accommodation_field")

    def close(self):
        if getattr(self, "h", None):
            load().lbm_adj_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self):
        """Runs the steps; returns (CL, light-species outlet flux)."""
        cl, fl = _D(), _D()
        _check(load().lbm_adj_forward(self.h, ctypes.byref(cl), ctypes.byref(fl)),
               "lbm_adj_forward")
        return cl.value, fl.value

    def state(self) -> np.ndarray:
        f = np.empty((2, 9, self.N, self.N_x), dtype=np.float64)
        _check(load().lbm_adj_state(self.h, _dptr(f), f.size), "lbm_adj_state")
        return f

    def gradient(self, objective: int = LBM_ADJ_CL) -> dict:
        th, kn = _D(), _D()
        da = np.empty(2 * self.N_x, dtype=np.float64)
        _check(load().lbm_adj_gradient(self.h, int(objective), ctypes.byref(th), ctypes.byref(kn),
                                       _dptr(da), da.size), "lbm_adj_gradient")
        return {"theta": th.value, "Kn_out": kn.value, "alpha": da.reshape(2, self.N_x)}
