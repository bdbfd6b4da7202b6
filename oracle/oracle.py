"""ctypes front-end of the FQNM CPU oracle (fqnm_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and
by bench.py's CPU-baseline leg, never by the library.  The C file is compiled
here with gcc (no FMA contraction) into oracle/_build/liboracle.so.

Every function takes and returns numpy arrays; integer states are int64.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fqnm_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "liboracle.so")

KINDS = {"linear_upwind": 0, "linear_lf": 1, "burgers_lf": 2,
         "burgers_eo": 3, "burgers_godunov": 4}
ROUNDING = {"half_even": 0, "half_away": 1, "floor": 2}
BOUNDARY = {"periodic": 0, "transmissive": 1}

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O2 -ffp-contract=off); returns the .so path."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    stale = (not os.path.exists(LIB)
             or os.path.getmtime(LIB) < os.path.getmtime(SRC))
    if force or stale:
        tmp = LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_d = C.c_double
_i = C.c_int
_l = C.c_int64


def _declare(L):
    L.orc_quantise.argtypes = [_f64p, _l, _d, _i, _i64p]
    L.orc_split_table.argtypes = [_i, _d, _d, _d, _d, _d, _i, _l, _l, _i64p, _i64p]
    L.orc_step_split.argtypes = [_i, _d, _d, _d, _d, _d, _i, _i, _i64p, _l, _l,
                                 C.POINTER(C.c_int64)]
    L.orc_step_split_faces.argtypes = [_i, _d, _d, _d, _d, _d, _i, _i, _i64p, _l, _l]
    L.orc_cone.argtypes = [_i, _d, _d, _d, _d, _d, _i, _i64p, _l, _l,
                           C.POINTER(C.c_int64)]
    L.orc_window.argtypes = [_i, _d, _d, _d, _d, _d, _i, _i64p, _l, _l, _i64p]
    L.orc_euler_window.argtypes = [_d, _f64p, _d, _d, _i, _i64p, _l, _i, _i, _l, _i64p]
    L.orc_two_point_phi.argtypes = [_i, _d, _d, _d, _d, _d, _i, _l, _l]
    L.orc_two_point_phi.restype = C.c_int64
    L.orc_step_two_point.argtypes = [_i, _d, _d, _d, _d, _d, _i, _i, _i64p, _l, _l]
    L.orc_invariants.argtypes = [_i64p, _l, C.c_void_p, _i, _i64p]
    L.orc_step_nd.argtypes = [_i, _d, _d, _d, _d, _d, _i, _i, _i64p, _i64p, _l]
    L.orc_level_entropy.argtypes = [_i64p, _l]
    L.orc_level_entropy.restype = _d
    L.orc_fv_step_f64.argtypes = [_i, _d, _d, _d, _d, _i, _f64p, _l, _l]
    L.orc_fv_step_f32.argtypes = [_i, _d, _d, _d, _d, _i, _f32p, _l, _l]
    L.orc_roe_flux.argtypes = [_d, _f64p, _f64p, _f64p]
    L.orc_roe_flux.restype = None
    L.orc_euler_roe_step.argtypes = [_d, _f64p, _d, _d, _i, _i64p, _l, _l, _i64p]
    L.orc_euler_fv_step_f64.argtypes = [_d, _d, _d, _f64p, _l, _l]
    L.orc_euler_roe_step_mask.argtypes = [_d, _f64p, _d, _d, _i, _i, _i64p, _f64p, _l, _l, _i64p]
    L.orc_riemann_star.argtypes = [_d] * 7 + [_f64p]
    L.orc_riemann_sample.argtypes = [_d] * 9 + [_f64p, _l, _f64p, _f64p, _f64p]
    L.orc_riemann_right_shock_speed.argtypes = [_d] * 7
    L.orc_riemann_right_shock_speed.restype = _d
    for name in ("orc_quantise", "orc_split_table", "orc_step_split", "orc_step_nd",
                 "orc_step_split_faces", "orc_cone", "orc_window", "orc_euler_window",
                 "orc_step_two_point",
                 "orc_invariants", "orc_fv_step_f64", "orc_fv_step_f32",
                 "orc_euler_roe_step", "orc_euler_fv_step_f64", "orc_euler_roe_step_mask",
                 "orc_riemann_star", "orc_riemann_sample"):
        getattr(L, name).restype = C.c_int


def _check(rc, what):
    if rc != 0:
        raise RuntimeError("oracle %s failed (rc=%d)" % (what, rc))


# --------------------------------------------------------------------------
# Scalar method
# --------------------------------------------------------------------------

def quantise(u, delta, rounding="half_even"):
    u = np.ascontiguousarray(u, dtype=np.float64)
    q = np.empty(u.shape[0], dtype=np.int64)
    _check(lib().orc_quantise(u, u.shape[0], delta, ROUNDING[rounding], q), "quantise")
    return q


def split_table(kind, delta, dx, dt, lo, count, a=0.0, alpha=0.0,
                rounding="half_even"):
    p = np.empty(count, dtype=np.int64)
    m = np.empty(count, dtype=np.int64)
    _check(lib().orc_split_table(KINDS[kind], a, alpha, delta, dx, dt,
                                 ROUNDING[rounding], lo, count, p, m), "table")
    return p, m


def step(q, kind, delta, dx, dt, steps, a=0.0, alpha=0.0,
         rounding="half_even", boundary="periodic", return_bflux=False):
    """Advance a copy of q by `steps` steps of eq. update_rule (cell form)."""
    q = np.array(q, dtype=np.int64, copy=True)
    bf = C.c_int64(0)
    _check(lib().orc_step_split(KINDS[kind], a, alpha, delta, dx, dt,
                                ROUNDING[rounding], BOUNDARY[boundary], q,
                                q.shape[0], steps, C.byref(bf)), "step")
    return (q, bf.value) if return_bflux else q


def step_nd(q, kind, delta, dx, dt, steps, a=0.0, alpha=0.0, rounding="half_even"):
    """Advance a copy of the periodic d-dimensional state q (numpy array of
    shape (nz, ny, nx), (ny, nx) or (nx,); x fastest) by `steps` steps of the
    directional composition (eq. nd_transfer_rule)."""
    q = np.array(q, dtype=np.int64, copy=True, order="C")
    dims = np.array(q.shape[::-1], dtype=np.int64)
    _check(lib().orc_step_nd(KINDS[kind], a, alpha, delta, dx, dt, ROUNDING[rounding],
                             q.ndim, dims, q.reshape(-1), steps), "step_nd")
    return q


def step_faces(q, kind, delta, dx, dt, steps, a=0.0, alpha=0.0,
               rounding="half_even", boundary="periodic"):
    """Same step written face by face (pairwise antisymmetric exchange)."""
    q = np.array(q, dtype=np.int64, copy=True)
    _check(lib().orc_step_split_faces(KINDS[kind], a, alpha, delta, dx, dt,
                                      ROUNDING[rounding], BOUNDARY[boundary], q,
                                      q.shape[0], steps), "step_faces")
    return q


def cone(q0, centre, steps, kind, delta, dx, dt, a=0.0, alpha=0.0,
         rounding="half_even"):
    """q_centre after `steps` periodic steps, from its dependency window only."""
    n = q0.shape[0]
    idx = (np.arange(centre - steps, centre + steps + 1) % n)
    w = np.ascontiguousarray(np.asarray(q0, dtype=np.int64)[idx])
    out = C.c_int64(0)
    _check(lib().orc_cone(KINDS[kind], a, alpha, delta, dx, dt,
                          ROUNDING[rounding], w, w.shape[0], steps,
                          C.byref(out)), "cone")
    return out.value


def _scalar_window_cut(q0, first, count, steps):
    n = q0.shape[0]
    idx = np.arange(first - steps, first + count + steps) % n
    return np.ascontiguousarray(np.asarray(q0, dtype=np.int64)[idx])


def _scalar_window_run(w, steps, kind, delta, dx, dt, a, alpha, rounding):
    out = np.empty(w.shape[0] - 2 * steps, dtype=np.int64)
    _check(lib().orc_window(KINDS[kind], a, alpha, delta, dx, dt, ROUNDING[rounding],
                            w, w.shape[0], steps, out), "window")
    return out


def window(q0, first, count, steps, kind, delta, dx, dt, a=0.0, alpha=0.0,
           rounding="half_even"):
    """Cells [first, first+count) (mod n) after `steps` periodic steps,
    from their dependency window of count + 2*steps cells only."""
    w = _scalar_window_cut(q0, first, count, steps)
    return _scalar_window_run(w, steps, kind, delta, dx, dt, a, alpha, rounding)


def _euler_window_cut(q0, first, count, steps):
    n = q0.shape[1]
    a = max(0, first - steps)
    b = min(n, first + count + steps)
    w = np.ascontiguousarray(np.asarray(q0, dtype=np.int64)[:, a:b])
    left, right = int(a == 0), int(b == n)
    lo = first - (a if left else a + steps)        # offset of `first` in the result
    return w, left, right, lo


def _euler_window_run(w, left, right, lo, count, steps, gamma, delta, dx, dt, rounding):
    L = w.shape[1]
    W = L - steps * (2 - left - right)
    out = np.empty((3, W), dtype=np.int64)
    _check(lib().orc_euler_window(gamma, np.asarray(delta, dtype=np.float64), dx, dt,
                                  ROUNDING[rounding], w.reshape(-1), L, left, right,
                                  steps, out.reshape(-1)), "euler_window")
    return np.ascontiguousarray(out[:, lo:lo + count])


def euler_window(q0, first, count, steps, gamma, delta, dx, dt, rounding="half_even"):
    """Cells [first, first+count) of the integer Euler state (3, n) after
    `steps` transmissive steps, from their dependency window only (clipped
    at the domain ends, where the ghost copy applies)."""
    w, left, right, lo = _euler_window_cut(q0, first, count, steps)
    return _euler_window_run(w, left, right, lo, count, steps, gamma, delta, dx, dt,
                             rounding)


def _window_job(job):
    kind, args = job
    if kind == "scalar":
        return _scalar_window_run(*args)
    return _euler_window_run(*args)


def _split(n, parts):
    edges = np.linspace(0, n, parts + 1).astype(np.int64)
    return [(int(a), int(b - a)) for a, b in zip(edges[:-1], edges[1:]) if b > a]


def _pool_map(jobs, procs):
    """Run window jobs in a spawned process pool (safe in a process that
    already holds a CUDA context: spawn starts fresh interpreters)."""
    import multiprocessing as mp
    import sys
    procs = max(1, min(procs or os.cpu_count() or 1, len(jobs)))
    main_file = getattr(sys.modules.get("__main__"), "__file__", None)
    if procs == 1 or not (main_file and os.path.exists(main_file)):
        # a spawned worker re-imports the main script; without one (an
        # interactive or stdin session) run the windows in this process
        return [_window_job(j) for j in jobs]
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(_window_job, jobs, chunksize=1)


def step_by_windows(q0, steps, kind, delta, dx, dt, a=0.0, alpha=0.0,
                    rounding="half_even", parts=0, procs=0):
    """The whole periodic state after `steps` steps, assembled from
    independent windows evaluated in parallel processes (each window is
    the plain cell form of eq. update_rule on its dependency window; see
    window()).  Same result as step(), bit for bit."""
    q0 = np.asarray(q0, dtype=np.int64)
    parts = parts or (os.cpu_count() or 1)
    jobs = [("scalar", (_scalar_window_cut(q0, f, c, steps), steps, kind, delta, dx, dt,
                        a, alpha, rounding))
            for f, c in _split(q0.shape[0], parts)]
    return np.concatenate(_pool_map(jobs, procs))


def euler_cells(q0, spans, steps, gamma, delta, dx, dt, rounding="half_even", procs=0):
    """The integer Euler state on the cell runs `spans` [(first, count), ...]
    after `steps` steps, each from its dependency window, in parallel
    processes.  Returns a list of (3, count) arrays."""
    q0 = np.asarray(q0, dtype=np.int64)
    jobs = []
    for f, c in spans:
        w, left, right, lo = _euler_window_cut(q0, f, c, steps)
        jobs.append(("euler", (w, left, right, lo, c, steps, gamma, delta, dx, dt, rounding)))
    return _pool_map(jobs, procs)


def euler_step_by_windows(q0, steps, gamma, delta, dx, dt, rounding="half_even",
                          parts=0, procs=0):
    """The whole Euler state after `steps` steps from parallel windows;
    equal to euler_step()'s state, bit for bit."""
    parts = parts or (os.cpu_count() or 1)
    spans = _split(np.asarray(q0).shape[1], parts)
    return np.concatenate(euler_cells(q0, spans, steps, gamma, delta, dx, dt, rounding,
                                      procs), axis=1)


def two_point_phi(kind, delta, dx, dt, qL, qR, a=0.0, alpha=0.0,
                  rounding="half_even"):
    return lib().orc_two_point_phi(KINDS[kind], a, alpha, delta, dx, dt,
                                   ROUNDING[rounding], int(qL), int(qR))


def step_two_point(q, kind, delta, dx, dt, steps, a=0.0, alpha=0.0,
                   rounding="half_even", boundary="periodic"):
    q = np.array(q, dtype=np.int64, copy=True)
    _check(lib().orc_step_two_point(KINDS[kind], a, alpha, delta, dx, dt,
                                    ROUNDING[rounding], BOUNDARY[boundary], q,
                                    q.shape[0], steps), "step_two_point")
    return q


def invariants(q, other=None, boundary="periodic"):
    """(mass, total variation, l1 distance to `other` or 0)."""
    q = np.ascontiguousarray(q, dtype=np.int64)
    out = np.zeros(3, dtype=np.int64)
    optr = None
    if other is not None:
        other = np.ascontiguousarray(other, dtype=np.int64)
        optr = other.ctypes.data_as(C.c_void_p)
    _check(lib().orc_invariants(q, q.shape[0], optr, BOUNDARY[boundary], out),
           "invariants")
    return int(out[0]), int(out[1]), int(out[2])


def level_entropy(q):
    q = np.ascontiguousarray(q, dtype=np.int64)
    return lib().orc_level_entropy(q, q.shape[0])


def fv_step(u, kind, dx, dt, steps, a=0.0, alpha=0.0, boundary="periodic",
            precision="f64"):
    if precision == "f64":
        u = np.array(u, dtype=np.float64, copy=True)
        _check(lib().orc_fv_step_f64(KINDS[kind], a, alpha, dx, dt,
                                     BOUNDARY[boundary], u, u.shape[0], steps), "fv64")
    else:
        u = np.array(u, dtype=np.float32, copy=True)
        _check(lib().orc_fv_step_f32(KINDS[kind], a, alpha, dx, dt,
                                     BOUNDARY[boundary], u, u.shape[0], steps), "fv32")
    return u


# --------------------------------------------------------------------------
# Euler / Roe
# --------------------------------------------------------------------------

def roe_flux(gamma, UL, UR):
    F = np.zeros(3, dtype=np.float64)
    lib().orc_roe_flux(gamma, np.ascontiguousarray(UL, dtype=np.float64),
                       np.ascontiguousarray(UR, dtype=np.float64), F)
    return F


def euler_step(q, gamma, delta, dx, dt, steps, rounding="half_even"):
    """q: (3, n) int64 SoA.  Returns (q_new, boundary_flux[3])."""
    q = np.array(q, dtype=np.int64, copy=True, order="C")
    n = q.shape[1]
    bf = np.zeros(3, dtype=np.int64)
    _check(lib().orc_euler_roe_step(gamma, np.asarray(delta, dtype=np.float64),
                                    dx, dt, ROUNDING[rounding], q.reshape(-1),
                                    n, steps, bf), "euler_step")
    return q, bf


def euler_step_mask(q, uf, mask, gamma, delta, dx, dt, steps, rounding="half_even"):
    """Quantise only the components in mask (1 rho, 2 m, 4 E); the others
    evolve in double.  q: (3, n) int64 (unmasked rows ignored), uf: (3, n)
    float64 (masked rows ignored).  Returns (q, uf, boundary_flux)."""
    q = np.array(q, dtype=np.int64, copy=True, order="C")
    uf = np.array(uf, dtype=np.float64, copy=True, order="C")
    n = q.shape[1]
    bf = np.zeros(3, dtype=np.int64)
    _check(lib().orc_euler_roe_step_mask(gamma, np.asarray(delta, dtype=np.float64), dx, dt,
                                         ROUNDING[rounding], mask, q.reshape(-1),
                                         uf.reshape(-1), n, steps, bf), "euler_step_mask")
    return q, uf, bf


def euler_fv_step(U, gamma, dx, dt, steps):
    U = np.array(U, dtype=np.float64, copy=True, order="C")
    _check(lib().orc_euler_fv_step_f64(gamma, dx, dt, U.reshape(-1), U.shape[1],
                                       steps), "euler_fv")
    return U


def riemann_star(gamma, left, right):
    st = np.zeros(4, dtype=np.float64)
    _check(lib().orc_riemann_star(gamma, *left, *right, st), "riemann_star")
    return st


def riemann_sample(gamma, left, right, x0, t, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    r = np.empty_like(x); u = np.empty_like(x); p = np.empty_like(x)
    _check(lib().orc_riemann_sample(gamma, *left, *right, x0, t, x, x.shape[0],
                                    r, u, p), "riemann_sample")
    return r, u, p


def riemann_right_shock_speed(gamma, left, right):
    return lib().orc_riemann_right_shock_speed(gamma, *left, *right)
