"""Python binding of libfqnm (include/fqnm.h): the same names, argument
marshalling only.

Every computation runs in the library's CUDA kernels.  There is no fallback:
if the shared library is missing or cannot be built, load() raises.

Host arrays are numpy arrays; device buffers are anything exposing a device
pointer (an int, or an object with .data_ptr() such as a torch tensor).
Every call raises FqnmError on a non-OK status.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))

FQNM_OK = 0
STATUS = {0: "FQNM_OK", -1: "FQNM_ERR_ARG", -2: "FQNM_ERR_CFL", -3: "FQNM_ERR_RANGE",
          -4: "FQNM_ERR_OVERFLOW", -5: "FQNM_ERR_OOM", -6: "FQNM_ERR_CUDA",
          -7: "FQNM_ERR_TIMEOUT", -8: "FQNM_ERR_STATE", -9: "FQNM_ERR_BUSY"}
FLUX = {"linear_upwind": 0, "linear_lf": 1, "burgers_lf": 2, "burgers_eo": 3,
        "burgers_godunov": 4,
        "table": 8, "euler_roe": 16}
ROUNDING = {"half_even": 0, "half_away": 1, "floor": 2}
BOUNDARY = {"periodic": 0, "transmissive": 1}
OPTION = {"kernel": 0, "layout": 1, "cells_per_thread": 2, "block": 3, "k": 4,
          "margin": 5, "closed_form": 6, "recover": 7, "autotune": 8, "graph": 9,
          "pdl": 10, "pack16": 11, "quantise_mask": 12, "nd_tile": 13, "verify": 14,
          "fp64": 15}


class FqnmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (STATUS.get(status, status), message))
        self.status = status


class fqnm_flux(C.Structure):
    _fields_ = [("kind", C.c_int), ("a", C.c_double), ("alpha", C.c_double),
                ("gamma", C.c_double), ("rounding", C.c_int)]


class fqnm_invariants_t(C.Structure):
    _fields_ = [("mass", C.c_int64 * 3), ("tv", C.c_int64 * 3), ("l1", C.c_int64 * 3),
                ("boundary_flux", C.c_int64 * 3), ("step", C.c_uint64),
                ("nvars", C.c_int32)]


class fqnm_rule_info(C.Structure):
    _fields_ = [("lo", C.c_int64), ("hi", C.c_int64), ("evaluator", C.c_int32),
                ("has_plus", C.c_int32), ("has_minus", C.c_int32),
                ("monotone", C.c_int32), ("num", C.c_int64), ("den", C.c_int64),
                ("closed_form_sign", C.c_int32), ("recoveries", C.c_int32)]


class fqnm_stats(C.Structure):
    _fields_ = [("launches", C.c_uint64), ("steps", C.c_uint64),
                ("cell_updates", C.c_uint64), ("kernel", C.c_int32),
                ("layout", C.c_int32), ("cells_per_thread", C.c_int32),
                ("block", C.c_int32), ("k", C.c_int32), ("graph", C.c_int32)]


class fqnm_level_stats_t(C.Structure):
    _fields_ = [("step", C.c_uint64), ("n_cells", C.c_int64), ("occupied_prev", C.c_int64),
                ("occupied", C.c_int64), ("S_prev", C.c_double), ("S", C.c_double),
                ("n_eff", C.c_double), ("rho", C.c_double), ("rho_level", C.c_int64),
                ("pairs", C.c_int64), ("moved", C.c_int64)]


class fqnm_problem_spec(C.Structure):
    _fields_ = [("flux", fqnm_flux), ("delta", C.c_double), ("dx", C.c_double),
                ("dt", C.c_double), ("boundary", C.c_int)]


_lib = None
_lock = threading.Lock()
_vp = C.c_void_p
_st = C.c_int

# name -> (restype, argtypes)
PROTOTYPES = {
    "fqnm_create": (_st, [C.POINTER(fqnm_flux), C.POINTER(C.c_double), C.c_double,
                          C.c_double, C.c_int, C.POINTER(_vp)]),
    "fqnm_create_custom": (_st, [_vp, _vp, _vp, C.c_double, C.c_double, C.c_double,
                                 C.c_double, C.c_int, C.c_int, C.POINTER(_vp)]),
    "fqnm_create_table": (_st, [_vp, _vp, C.c_int64, C.c_int64, C.c_double, C.c_int,
                                C.POINTER(_vp)]),
    "fqnm_destroy": (_st, [_vp]),
    "fqnm_set_stream": (_st, [_vp, _vp]),
    "fqnm_set_option": (_st, [_vp, C.c_int, C.c_int64]),
    "fqnm_quantise": (_st, [_vp, C.c_size_t, C.c_double, C.c_int, C.c_int, _vp]),
    "fqnm_quantise_device": (_st, [_vp, C.c_size_t, C.c_double, C.c_int, C.c_int, _vp, _vp]),
    "fqnm_load_states": (_st, [_vp, _vp, C.c_size_t]),
    "fqnm_load_states_device": (_st, [_vp, _vp, C.c_size_t]),
    "fqnm_load_field": (_st, [_vp, _vp, C.c_size_t, C.c_int]),
    "fqnm_step": (_st, [_vp, C.c_uint64]),
    "fqnm_sync": (_st, [_vp]),
    "fqnm_observe": (_st, [_vp, _vp]),
    "fqnm_observe_device": (_st, [_vp, _vp, C.c_int]),
    "fqnm_checkpoint": (_st, [_vp, _vp, C.POINTER(C.c_uint64)]),
    "fqnm_checkpoint_device": (_st, [_vp, _vp]),
    "fqnm_invariants": (_st, [_vp, _vp, C.POINTER(fqnm_invariants_t)]),
    "fqnm_invariants_noalloc": (_st, [_vp, _vp, C.c_size_t, C.c_int,
                                      C.POINTER(C.c_int64), _vp]),
    "fqnm_fp64_check": (_st, [C.c_int, C.c_int, _vp, _vp, C.c_size_t, _vp, _vp, _vp, _vp]),
    "fqnm_get_size": (_st, [_vp, C.POINTER(C.c_size_t), C.POINTER(C.c_int)]),
    "fqnm_set_grid": (_st, [_vp, C.c_int, C.POINTER(C.c_size_t)]),
    "fqnm_resume": (_st, [_vp, _vp, C.c_size_t, C.c_uint64, C.POINTER(C.c_int64)]),
    "fqnm_state_device": (_st, [_vp, C.POINTER(_vp), C.POINTER(C.c_size_t)]),
    "fqnm_hopf_lax": (_st, [_vp, C.c_size_t, _vp, _vp, C.c_size_t, C.c_double, _vp, _vp,
                            C.c_int, _vp]),
    "fqnm_level_step": (_st, [_vp, C.POINTER(fqnm_level_stats_t)]),
    "fqnm_level_series": (_st, [_vp, C.c_uint64, C.c_uint64, C.POINTER(fqnm_level_stats_t)]),
    "fqnm_level_transitions": (_st, [_vp, _vp, _vp, _vp, C.c_size_t, C.POINTER(C.c_size_t)]),
    "fqnm_level_histogram": (_st, [_vp, C.POINTER(C.c_int64), _vp, C.c_size_t,
                                   C.POINTER(C.c_size_t)]),
    "fqnm_get_rule": (_st, [_vp, C.POINTER(fqnm_rule_info)]),
    "fqnm_get_tables": (_st, [_vp, _vp, _vp]),
    "fqnm_get_stats": (_st, [_vp, C.POINTER(fqnm_stats), C.c_int]),
    "fqnm_fv_create": (_st, [C.POINTER(fqnm_flux), C.c_double, C.c_double, C.c_int,
                             C.c_int, C.POINTER(_vp)]),
    "fqnm_fv_destroy": (_st, [_vp]),
    "fqnm_fv_set_stream": (_st, [_vp, _vp]),
    "fqnm_fv_load": (_st, [_vp, _vp, C.c_size_t]),
    "fqnm_fv_load_device": (_st, [_vp, _vp, C.c_size_t]),
    "fqnm_fv_step": (_st, [_vp, C.c_uint64]),
    "fqnm_fv_set_k": (_st, [_vp, C.c_int]),
    "fqnm_fv_observe": (_st, [_vp, _vp]),
    "fqnm_fv_observe_device": (_st, [_vp, _vp]),
    "fqnm_fv_launches": (_st, [_vp, C.POINTER(C.c_uint64)]),
    "fqnm_fv_get_size": (_st, [_vp, C.POINTER(C.c_size_t), C.POINTER(C.c_int)]),
    "fqnm_batch_create": (_st, [C.c_size_t, C.c_int, _vp, C.POINTER(_vp)]),
    "fqnm_batch_destroy": (_st, [_vp]),
    "fqnm_batch_set_plan": (_st, [_vp, C.c_int, C.c_int, C.c_int, C.c_int]),
    "fqnm_batch_autotune": (_st, [_vp, C.c_int]),
    "fqnm_batch_set_margin": (_st, [_vp, C.c_int64]),
    "fqnm_batch_get_plan": (_st, [_vp] + [C.POINTER(C.c_int)] * 5),
    "fqnm_batch_submit": (_st, [_vp, C.POINTER(fqnm_problem_spec), _vp, C.c_size_t,
                                C.c_uint64, C.c_uint64, C.POINTER(C.c_int64)]),
    "fqnm_batch_progress": (_st, [_vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "fqnm_batch_poll": (_st, [_vp, C.c_int64, _vp, C.c_size_t, C.POINTER(C.c_uint64),
                              C.POINTER(C.c_int)]),
    "fqnm_batch_completed": (_st, [_vp, C.POINTER(C.c_int64), C.c_int, C.POINTER(C.c_int)]),
    "fqnm_batch_submit_device": (_st, [_vp, C.POINTER(fqnm_problem_spec), _vp, C.c_size_t,
                                       C.c_uint64, C.c_uint64, _vp, C.POINTER(C.c_int64)]),
    "fqnm_batch_stats": (_st, [_vp, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64),
                               C.POINTER(C.c_uint64), C.POINTER(C.c_double)]),
    "fqnm_clock_ns": (C.c_uint64, []),
    "fqnm_last_error": (C.c_char_p, []),
    "fqnm_status_string": (C.c_char_p, [C.c_int]),
    "fqnm_version": (C.c_int, []),
    "fqnm_kernel_launches": (C.c_uint64, []),
}


def lib_path(checked: bool = False) -> str:
    return os.path.join(HERE, "_build", "libfqnm_checked.so" if checked else "libfqnm.so")


def checked_build() -> bool:
    """FQNM_CHECKED=1 selects the checked library (computed indices verified
    before each access; a bad one is reported as FQNM_ERR_STATE)."""
    return os.environ.get("FQNM_CHECKED") == "1"


def load(build: bool = True):
    """Load libfqnm (building it in-tree first if its sources changed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path(checked_build())
        if build:
            from . import build as _b
            path = _b.build(checked=checked_build())
        if not os.path.exists(path):
            raise FqnmError(-6, "libfqnm is not built (%s); run build()" % path)
        L = C.CDLL(path)
        for name, (res, args) in PROTOTYPES.items():
            fn = getattr(L, name, None)
            if fn is None:
                continue
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def _check(st: int):
    if st != FQNM_OK:
        msg = load().fqnm_last_error()
        raise FqnmError(st, msg.decode() if msg else "")


def _dptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError("need a device pointer (int) or an object with data_ptr()")


def _stream(s) -> Optional[int]:
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return getattr(s, "cuda_stream", None) or getattr(s, "ptr", None)


def make_flux(kind: str, a: float = 0.0, alpha: float = 0.0, gamma: float = 0.0,
              rounding: str = "half_even") -> fqnm_flux:
    return fqnm_flux(FLUX[kind], a, alpha, gamma, ROUNDING[rounding])


# ---------------------------------------------------------------------------
# solver calls (same names as the C ABI)
# ---------------------------------------------------------------------------

def fqnm_create(flux: fqnm_flux, delta, dx: float, dt: float,
                boundary: str = "periodic") -> int:
    d = np.atleast_1d(np.asarray(delta, dtype=np.float64))
    out = _vp()
    _check(load().fqnm_create(C.byref(flux), d.ctypes.data_as(C.POINTER(C.c_double)),
                              dx, dt, BOUNDARY[boundary], C.byref(out)))
    return out.value


def fqnm_create_table(phi_p, phi_m, lo: int, delta: float,
                      boundary: str = "periodic") -> int:
    p = np.ascontiguousarray(phi_p, dtype=np.int32)
    m = np.ascontiguousarray(phi_m, dtype=np.int32)
    if p.shape != m.shape:
        raise ValueError("phi_p and phi_m differ in length")
    out = _vp()
    _check(load().fqnm_create_table(p.ctypes.data, m.ctypes.data, lo, p.shape[0], delta,
                                    BOUNDARY[boundary], C.byref(out)))
    return out.value


def fqnm_destroy(h: int):
    _check(load().fqnm_destroy(h))


def fqnm_set_stream(h: int, stream=None):
    _check(load().fqnm_set_stream(h, _stream(stream)))


def fqnm_set_option(h: int, option: str, value: int):
    _check(load().fqnm_set_option(h, OPTION[option], int(value)))


def fqnm_quantise(u, delta: float, rounding: str = "half_even", state_bits: int = 32):
    u = np.ascontiguousarray(u, dtype=np.float64)
    q = np.empty(u.shape[0], dtype=np.int32 if state_bits == 32 else np.int64)
    _check(load().fqnm_quantise(u.ctypes.data, u.shape[0], delta, ROUNDING[rounding],
                                state_bits, q.ctypes.data))
    return q


def fqnm_quantise_device(u_dev, n: int, delta: float, q_dev, rounding: str = "half_even",
                         state_bits: int = 32, stream=None):
    _check(load().fqnm_quantise_device(_dptr(u_dev), n, delta, ROUNDING[rounding],
                                       state_bits, _dptr(q_dev), _stream(stream)))


def fqnm_load_states(h: int, q, nvars: Optional[int] = None):
    hv = fqnm_get_size(h)[1]
    if nvars is not None and nvars != hv:
        raise ValueError("the solver has %d variables" % hv)
    nvars = hv
    q = np.ascontiguousarray(q, dtype=np.int32 if nvars == 1 else np.int64)
    n = q.shape[-1] if q.ndim > 1 else q.shape[0]
    if q.size != nvars * n:
        raise ValueError("states must be [%d][n]" % nvars)
    _check(load().fqnm_load_states(h, q.ctypes.data, n))


def fqnm_load_states_device(h: int, q_dev, n_cells: int):
    _check(load().fqnm_load_states_device(h, _dptr(q_dev), n_cells))


def fqnm_load_field(h: int, u, n_cells: Optional[int] = None, on_device: bool = False):
    """u: numpy [nvars][n] doubles (host) or a device pointer with n_cells."""
    if on_device:
        _check(load().fqnm_load_field(h, _dptr(u), n_cells, 1))
        return
    u = np.ascontiguousarray(u, dtype=np.float64)
    nvars = fqnm_get_size(h)[1]
    if u.size != nvars * u.shape[-1]:
        raise ValueError("field must be [%d][n] doubles" % nvars)
    _check(load().fqnm_load_field(h, u.ctypes.data, u.shape[-1], 0))


def fqnm_step(h: int, k: int):
    _check(load().fqnm_step(h, k))


def fqnm_sync(h: int):
    _check(load().fqnm_sync(h))


def fqnm_get_size(h: int):
    """(cells, conserved variables) of the loaded state."""
    n, nv = C.c_size_t(0), C.c_int(0)
    _check(load().fqnm_get_size(h, C.byref(n), C.byref(nv)))
    return n.value, nv.value


def _host_size(h: int, n: Optional[int], nvars: Optional[int]):
    """The handle's own size; a caller's n / nvars must agree with it (the
    library writes that many values into the host buffer)."""
    hn, hv = fqnm_get_size(h)
    if hn == 0:
        raise FqnmError(-8, "no state loaded")
    if (n is not None and n != hn) or (nvars is not None and nvars != hv):
        raise ValueError("size (%s, %s) does not match the loaded state (%d, %d)"
                         % (n, nvars, hn, hv))
    return hn, hv


def fqnm_observe(h: int, n: Optional[int] = None, nvars: Optional[int] = None) -> np.ndarray:
    n, nvars = _host_size(h, n, nvars)
    u = np.empty(n * nvars, dtype=np.float64)
    _check(load().fqnm_observe(h, u.ctypes.data))
    return u.reshape(nvars, n) if nvars > 1 else u


def fqnm_observe_device(h: int, u_dev, fp32: bool = False):
    _check(load().fqnm_observe_device(h, _dptr(u_dev), 1 if fp32 else 0))


def fqnm_checkpoint(h: int, n: Optional[int] = None, nvars: Optional[int] = None):
    n, nvars = _host_size(h, n, nvars)
    q = np.empty(n * nvars, dtype=np.int32 if nvars == 1 else np.int64)
    step = C.c_uint64(0)
    _check(load().fqnm_checkpoint(h, q.ctypes.data, C.byref(step)))
    return (q.reshape(nvars, n) if nvars > 1 else q), step.value


def fqnm_checkpoint_device(h: int, q_dev):
    _check(load().fqnm_checkpoint_device(h, _dptr(q_dev)))


def fqnm_invariants(h: int, other: Optional[int] = None) -> dict:
    out = fqnm_invariants_t()
    _check(load().fqnm_invariants(h, other or None, C.byref(out)))
    nv = out.nvars
    return {"mass": list(out.mass)[:nv], "tv": list(out.tv)[:nv], "l1": list(out.l1)[:nv],
            "boundary_flux": list(out.boundary_flux)[:nv], "step": out.step}


def fqnm_invariants_noalloc(q_dev, n: int, other_dev=None, boundary: str = "periodic",
                            stream=None) -> tuple:
    """(mass, total variation, l1) of a device int32 state, computed with the
    library's static scratch array: no device allocation per call."""
    out = (C.c_int64 * 3)()
    _check(load().fqnm_invariants_noalloc(_dptr(q_dev), _dptr(other_dev) or None, n,
                                          BOUNDARY[boundary], out, _stream(stream)))
    return out[0], out[1], out[2]


def fqnm_fp64_check(op: int, a_dev, b_dev, n: int, out_int, out_fp64, out_path,
                    rounding: str = "half_even", stream=None):
    """The integer-pipe IEEE double step `op` (0 divide, 1 square root,
    2 scaled int64 conversion, 3 scaled rounding to int64) next to the FP64
    instruction, on device arrays (see include/fqnm.h)."""
    _check(load().fqnm_fp64_check(int(op), ROUNDING[rounding], _dptr(a_dev), _dptr(b_dev), n,
                                  _dptr(out_int), _dptr(out_fp64), _dptr(out_path),
                                  _stream(stream)))


def fqnm_resume(h: int, q, step: int, boundary_flux=None, nvars: Optional[int] = None):
    """Load checkpointed states and continue at `step` with the given boundary
    transfer totals (as returned by fqnm_invariants)."""
    hv = fqnm_get_size(h)[1]
    q = np.ascontiguousarray(q, dtype=np.int32 if hv == 1 else np.int64)
    n = q.shape[-1] if q.ndim > 1 else q.shape[0]
    if q.size != hv * n:
        raise ValueError("states must be [%d][n]" % hv)
    bf = None
    if boundary_flux is not None:
        bf = (C.c_int64 * 3)(*[int(v) for v in list(boundary_flux)[:hv]])
    _check(load().fqnm_resume(h, q.ctypes.data, n, int(step), bf))


def fqnm_state_device(h: int):
    """(device pointer, cells) of the live state."""
    ptr = _vp()
    n = C.c_size_t(0)
    _check(load().fqnm_state_device(h, C.byref(ptr), C.byref(n)))
    return ptr.value, n.value


def fqnm_set_grid(h: int, dims) -> None:
    """dims in x-fastest order, e.g. (nx, ny) or (nx, ny, nz)."""
    arr = (C.c_size_t * 3)(*([int(v) for v in dims] + [1] * (3 - len(dims))))
    _check(load().fqnm_set_grid(h, len(dims), arr))


def fqnm_hopf_lax(x, y, U0y, t: float, nx: Optional[int] = None, ny: Optional[int] = None,
                  u=None, idx=None, stream=None):
    """Hopf-Lax entropy solution of Burgers at the points x from candidates
    (y, U0(y)).  Host numpy arrays: returns (u, idx).  Device pointers (with
    nx, ny and output pointers u, idx): enqueued on `stream`, returns None."""
    if nx is not None:
        _check(load().fqnm_hopf_lax(_dptr(x), nx, _dptr(y), _dptr(U0y), ny, t, _dptr(u),
                                    _dptr(idx) or None, 1, _stream(stream)))
        return None
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    U0y = np.ascontiguousarray(U0y, dtype=np.float64)
    if y.shape != U0y.shape:
        raise ValueError("y and U0y differ in size")
    u = np.empty(x.size, dtype=np.float64)
    idx = np.empty(x.size, dtype=np.int64)
    _check(load().fqnm_hopf_lax(x.ctypes.data, x.size, y.ctypes.data, U0y.ctypes.data, y.size,
                                t, u.ctypes.data, idx.ctypes.data, 0, None))
    return u, idx


def _level_dict(r: fqnm_level_stats_t) -> dict:
    return {f: getattr(r, f) for f, _ in fqnm_level_stats_t._fields_}


def fqnm_level_step(h: int) -> dict:
    """One step and the level statistics of that transition (entropy appendix)."""
    out = fqnm_level_stats_t()
    _check(load().fqnm_level_step(h, C.byref(out)))
    return _level_dict(out)


def fqnm_level_series(h: int, records: int, every: int) -> list:
    out = (fqnm_level_stats_t * max(records, 1))()
    _check(load().fqnm_level_series(h, records, every, out))
    return [_level_dict(out[r]) for r in range(records)]


def fqnm_level_transitions(h: int):
    """(k, k_next, count) int64 arrays: the nonzero N_{k'k} of the last
    recorded transition, sorted by k then k'."""
    m = C.c_size_t(0)
    st = load().fqnm_level_transitions(h, None, None, None, 0, C.byref(m))
    if st != FQNM_OK and m.value == 0:
        _check(st)
    k = np.empty(m.value, dtype=np.int64)
    kn = np.empty(m.value, dtype=np.int64)
    cnt = np.empty(m.value, dtype=np.int64)
    _check(load().fqnm_level_transitions(h, k.ctypes.data, kn.ctypes.data, cnt.ctypes.data,
                                         m.value, C.byref(m)))
    return k, kn, cnt


def fqnm_level_histogram(h: int):
    """(lo, counts): dense level counts of the current state from its min."""
    lo = C.c_int64(0)
    n = C.c_size_t(0)
    st = load().fqnm_level_histogram(h, C.byref(lo), None, 0, C.byref(n))
    if st != FQNM_OK and n.value == 0:
        _check(st)
    counts = np.empty(n.value, dtype=np.int64)
    _check(load().fqnm_level_histogram(h, C.byref(lo), counts.ctypes.data, n.value,
                                       C.byref(n)))
    return lo.value, counts


def fqnm_get_rule(h: int) -> dict:
    out = fqnm_rule_info()
    _check(load().fqnm_get_rule(h, C.byref(out)))
    return {f: getattr(out, f) for f, _ in fqnm_rule_info._fields_}


def fqnm_get_tables(h: int):
    r = fqnm_get_rule(h)
    cnt = r["hi"] - r["lo"] + 1
    p = np.empty(cnt, dtype=np.int32)
    m = np.empty(cnt, dtype=np.int32)
    _check(load().fqnm_get_tables(h, p.ctypes.data, m.ctypes.data))
    return r["lo"], p, m


def fqnm_get_stats(h: int, reset: bool = False) -> dict:
    out = fqnm_stats()
    _check(load().fqnm_get_stats(h, C.byref(out), 1 if reset else 0))
    return {f: getattr(out, f) for f, _ in fqnm_stats._fields_}


# ---------------------------------------------------------------------------
# finite-volume baseline
# ---------------------------------------------------------------------------

def fqnm_fv_create(flux: fqnm_flux, dx: float, dt: float, boundary: str = "periodic",
                   precision: int = 64) -> int:
    out = _vp()
    _check(load().fqnm_fv_create(C.byref(flux), dx, dt, BOUNDARY[boundary], precision,
                                 C.byref(out)))
    return out.value


def fqnm_fv_destroy(h: int):
    _check(load().fqnm_fv_destroy(h))


def fqnm_fv_set_stream(h: int, stream=None):
    _check(load().fqnm_fv_set_stream(h, _stream(stream)))


def fqnm_fv_load(h: int, u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    n = u.shape[-1]
    nvars = fqnm_fv_get_size(h)[1]
    if u.size != nvars * n:
        raise ValueError("field must be [%d][n] doubles" % nvars)
    _check(load().fqnm_fv_load(h, u.ctypes.data, n))


def fqnm_fv_load_device(h: int, u_dev, n_cells: int):
    _check(load().fqnm_fv_load_device(h, _dptr(u_dev), n_cells))


def fqnm_fv_step(h: int, k: int):
    _check(load().fqnm_fv_step(h, k))


def fqnm_fv_set_k(h: int, k: int):
    _check(load().fqnm_fv_set_k(h, k))


def fqnm_fv_get_size(h: int):
    n, nv = C.c_size_t(0), C.c_int(0)
    _check(load().fqnm_fv_get_size(h, C.byref(n), C.byref(nv)))
    return n.value, nv.value


def fqnm_fv_observe(h: int, n: Optional[int] = None, nvars: Optional[int] = None) -> np.ndarray:
    hn, hv = fqnm_fv_get_size(h)
    if hn == 0:
        raise FqnmError(-8, "no field loaded")
    if (n is not None and n != hn) or (nvars is not None and nvars != hv):
        raise ValueError("size (%s, %s) does not match the loaded field (%d, %d)"
                         % (n, nvars, hn, hv))
    n, nvars = hn, hv
    u = np.empty(n * nvars, dtype=np.float64)
    _check(load().fqnm_fv_observe(h, u.ctypes.data))
    return u.reshape(nvars, n) if nvars > 1 else u


def fqnm_fv_observe_device(h: int, u_dev):
    _check(load().fqnm_fv_observe_device(h, _dptr(u_dev)))


def fqnm_fv_launches(h: int) -> int:
    v = C.c_uint64(0)
    _check(load().fqnm_fv_launches(h, C.byref(v)))
    return v.value


# ---------------------------------------------------------------------------
# batched serving
# ---------------------------------------------------------------------------

def make_spec(p) -> fqnm_problem_spec:
    """Problem spec for an inputs.ScalarProblem."""
    return fqnm_problem_spec(make_flux(p.flux, a=p.a, alpha=p.alpha), p.delta, p.dx, p.dt,
                             BOUNDARY[p.boundary])


def fqnm_batch_create(mem_budget_bytes: int, max_slots: int, stream=None) -> int:
    out = _vp()
    _check(load().fqnm_batch_create(mem_budget_bytes, max_slots, _stream(stream), C.byref(out)))
    return out.value


def fqnm_batch_destroy(b: int):
    _check(load().fqnm_batch_destroy(b))


def fqnm_batch_set_plan(b: int, cells_per_thread: int = 0, block: int = 0, k: int = 0,
                        layout: int = 0):
    _check(load().fqnm_batch_set_plan(b, cells_per_thread, block, k, layout))


def fqnm_batch_autotune(b: int, epochs_per_plan: int = 3):
    _check(load().fqnm_batch_autotune(b, epochs_per_plan))


def fqnm_batch_set_margin(b: int, margin: int):
    _check(load().fqnm_batch_set_margin(b, int(margin)))


def fqnm_batch_get_plan(b: int) -> dict:
    v = [C.c_int(0) for _ in range(5)]
    _check(load().fqnm_batch_get_plan(b, *[C.byref(x) for x in v]))
    return dict(zip(("cells_per_thread", "block", "k", "layout", "tuning"), [x.value for x in v]))


def fqnm_batch_submit(b: int, spec: fqnm_problem_spec, q0, steps: int,
                      arrival_ns: int = 0) -> int:
    q = np.ascontiguousarray(q0, dtype=np.int32)
    rid = C.c_int64(0)
    _check(load().fqnm_batch_submit(b, C.byref(spec), q.ctypes.data, q.shape[0], steps,
                                    arrival_ns, C.byref(rid)))
    return rid.value


def fqnm_batch_submit_device(b: int, spec: fqnm_problem_spec, q0_dev, n: int, steps: int,
                             arrival_ns: int = 0, out_dev=None) -> int:
    rid = C.c_int64(0)
    _check(load().fqnm_batch_submit_device(b, C.byref(spec), _dptr(q0_dev), n, steps,
                                           arrival_ns, _dptr(out_dev) or None, C.byref(rid)))
    return rid.value


def fqnm_batch_progress(b: int, max_epochs: int = 1):
    a, q = C.c_int(0), C.c_int(0)
    _check(load().fqnm_batch_progress(b, max_epochs, C.byref(a), C.byref(q)))
    return a.value, q.value


def fqnm_batch_poll(b: int, rid: int, n: int):
    """(state or None, latency_ns) -- the state is released on success."""
    q = np.empty(n, dtype=np.int32)
    lat, done = C.c_uint64(0), C.c_int(0)
    _check(load().fqnm_batch_poll(b, rid, q.ctypes.data, n, C.byref(lat), C.byref(done)))
    return (q, lat.value) if done.value else (None, 0)


def fqnm_batch_completed(b: int, max_ids: int = 4096):
    ids = (C.c_int64 * max_ids)()
    n = C.c_int(0)
    _check(load().fqnm_batch_completed(b, ids, max_ids, C.byref(n)))
    return list(ids[:n.value])


def fqnm_batch_stats(b: int) -> dict:
    l, c, e, g = C.c_uint64(0), C.c_uint64(0), C.c_uint64(0), C.c_double(0)
    _check(load().fqnm_batch_stats(b, C.byref(l), C.byref(c), C.byref(e), C.byref(g)))
    return {"launches": l.value, "cell_updates": c.value, "epochs": e.value,
            "gpu_ms": g.value}


def fqnm_clock_ns() -> int:
    return load().fqnm_clock_ns()


def fqnm_last_error() -> str:
    m = load().fqnm_last_error()
    return m.decode() if m else ""


def fqnm_version() -> int:
    return load().fqnm_version()


def fqnm_kernel_launches() -> int:
    return load().fqnm_kernel_launches()


# ---------------------------------------------------------------------------
# small convenience wrapper (still marshalling only)
# ---------------------------------------------------------------------------

SPLIT_FN = C.CFUNCTYPE(C.c_double, C.c_double, C.c_void_p)


def fqnm_create_custom(fplus, fminus, alpha: float, delta: float, dx: float, dt: float,
                       boundary: str = "periodic", rounding: str = "half_even"):
    """A solver for a custom monotone split given as Python callables of u.
    Returns (handle, callbacks); keep the callbacks alive with the handle."""
    cbs = (SPLIT_FN(lambda u, _: fplus(u)), SPLIT_FN(lambda u, _: fminus(u)))
    h = _vp()
    _check(load().fqnm_create_custom(C.cast(cbs[0], _vp), C.cast(cbs[1], _vp), None, alpha,
                                     delta, dx, dt, BOUNDARY[boundary], ROUNDING[rounding],
                                     C.byref(h)))
    return h.value, cbs


class Solver:
    """Owns one fqnm_solver handle; methods call the functions above."""

    def __init__(self, flux: fqnm_flux, delta, dx: float, dt: float,
                 boundary: str = "periodic", **options):
        self.nvars = 3 if flux.kind == FLUX["euler_roe"] else 1
        self.h = fqnm_create(flux, delta, dx, dt, boundary)
        self.n = 0
        for k, v in options.items():
            fqnm_set_option(self.h, k, v)

    @classmethod
    def custom(cls, fplus, fminus, alpha: float, delta: float, dx: float, dt: float,
               boundary: str = "periodic", rounding: str = "half_even", **options):
        """Solver for host callables f+(u), f-(u) (tabulated at load)."""
        self = cls.__new__(cls)
        self.nvars = 1
        self.h, self._callbacks = fqnm_create_custom(fplus, fminus, alpha, delta, dx, dt,
                                                     boundary, rounding)
        self.n = 0
        for k, v in options.items():
            fqnm_set_option(self.h, k, v)
        return self

    @classmethod
    def for_problem(cls, p, rounding: str = "half_even", **options):
        """Solver for an inputs.ScalarProblem."""
        flux = make_flux(p.flux, a=p.a, alpha=p.alpha, rounding=rounding)
        return cls(flux, p.delta, p.dx, p.dt, p.boundary, **options)

    def load(self, q):
        q = np.asarray(q)
        self.n = q.shape[-1]
        fqnm_load_states(self.h, q, self.nvars)
        return self

    def load_device(self, q_dev, n):
        self.n = n
        fqnm_load_states_device(self.h, q_dev, n)
        return self

    def load_field(self, u, n=None, on_device=False):
        """Quantise a double field (host array, or device pointer with n)."""
        fqnm_load_field(self.h, u, n, on_device)
        self.n = fqnm_get_size(self.h)[0]
        return self

    def step(self, k: int):
        fqnm_step(self.h, k)
        return self

    def state(self):
        return fqnm_checkpoint(self.h)[0]

    def observe(self):
        return fqnm_observe(self.h)

    def invariants(self, other: Optional["Solver"] = None):
        return fqnm_invariants(self.h, other.h if other else None)

    def set_grid(self, dims):
        """Periodic Cartesian grid, dims x-fastest (call before load)."""
        fqnm_set_grid(self.h, dims)
        return self

    def level_step(self) -> dict:
        return fqnm_level_step(self.h)

    def level_series(self, records: int, every: int) -> list:
        return fqnm_level_series(self.h, records, every)

    def level_transitions(self):
        return fqnm_level_transitions(self.h)

    def level_histogram(self):
        return fqnm_level_histogram(self.h)

    def rule(self):
        return fqnm_get_rule(self.h)

    def stats(self, reset=False):
        return fqnm_get_stats(self.h, reset)

    def close(self):
        if self.h:
            fqnm_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
