"""The C ABI without a GPU: the library builds, loads, exports every function
include/fqnm.h declares, and validates arguments on the host."""
import os
import re

import numpy as np
import pytest

from paper_2604_06947_gb300 import fqnm as F
from paper_2604_06947_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*"
                            r"(fqnm_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_core_calls():
    names = declared_functions()
    for must in ("fqnm_create", "fqnm_load_states", "fqnm_step", "fqnm_observe",
                 "fqnm_invariants", "fqnm_destroy", "fqnm_fv_create"):
        assert must in names


def test_library_exports_every_declared_symbol(fq):
    L = fq.load()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    # and the binding knows every one of them
    assert set(declared_functions()) <= set(F.PROTOTYPES), \
        set(declared_functions()) - set(F.PROTOTYPES)


def test_version_and_status_strings(fq):
    assert F.fqnm_version() >= 100
    assert F.load().fqnm_status_string(-2) == b"Courant number above 1"


def test_create_validates_on_host(fq):
    p = I.linear_advection_problem(with_u0=False)
    h = F.fqnm_create(F.make_flux("linear_upwind", a=1.0), p.delta, p.dx, p.dt)
    F.fqnm_destroy(h)
    with pytest.raises(F.FqnmError) as e:       # nu = 1.5
        F.fqnm_create(F.make_flux("linear_upwind", a=1.0), p.delta, p.dx, 1.5 * p.dx)
    assert e.value.status == -2
    with pytest.raises(F.FqnmError) as e:       # delta not a power of two
        F.fqnm_create(F.make_flux("linear_upwind", a=1.0), 0.001, p.dx, p.dt)
    assert e.value.status == -1
    with pytest.raises(F.FqnmError) as e:       # LF needs alpha >= |a|
        F.fqnm_create(F.make_flux("linear_lf", a=1.0, alpha=0.5), p.delta, p.dx, p.dt)
    assert e.value.status == -1
    with pytest.raises(F.FqnmError) as e:       # Euler needs transmissive ends
        F.fqnm_create(F.make_flux("euler_roe", gamma=1.4), [2.0 ** -32] * 3, 0.01, 0.001,
                      "periodic")
    assert e.value.status == -1
    # the CFL limit itself is accepted (nu = 1)
    F.fqnm_destroy(F.fqnm_create(F.make_flux("burgers_lf", alpha=1.3), 2.0 ** -16, 0.01,
                                 0.01 / 1.3))


def test_calls_out_of_order(fq):
    h = F.fqnm_create(F.make_flux("linear_upwind", a=1.0), 2.0 ** -10, 0.01, 0.005)
    with pytest.raises(F.FqnmError) as e:
        F.fqnm_step(h, 1)
    assert e.value.status == -8
    with pytest.raises(F.FqnmError) as e:
        F.fqnm_set_option(h, "cells_per_thread", 5)
    assert e.value.status == -1
    F.fqnm_destroy(h)


def test_option_bounds(fq):
    """Option values outside their sets are refused before any GPU work:
    kernel 3 (the Euler kernel's number, not a plan), K of the FV baseline
    outside 1..64, K > 1 on transmissive ends."""
    h = F.fqnm_create(F.make_flux("linear_upwind", a=1.0), 2.0 ** -10, 0.01, 0.005)
    for bad in (-1, 3, 5):
        with pytest.raises(F.FqnmError) as e:
            F.fqnm_set_option(h, "kernel", bad)
        assert e.value.status == -1
    for ok in (0, 1, 2, 4):
        F.fqnm_set_option(h, "kernel", ok)
    F.fqnm_destroy(h)
    fv = F.fqnm_fv_create(F.make_flux("linear_upwind", a=1.0), 0.01, 0.005, "periodic", 32)
    for bad in (0, 65):
        with pytest.raises(F.FqnmError) as e:
            F.fqnm_fv_set_k(fv, bad)
        assert e.value.status == -1
    F.fqnm_fv_set_k(fv, 64)
    F.fqnm_fv_destroy(fv)
    fv = F.fqnm_fv_create(F.make_flux("linear_upwind", a=1.0), 0.01, 0.005, "transmissive", 64)
    with pytest.raises(F.FqnmError):
        F.fqnm_fv_set_k(fv, 2)
    F.fqnm_fv_destroy(fv)


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.mark.skipif(_has_gpu(), reason="checks the no-GPU error path")
def test_no_gpu_is_a_status_not_a_crash(fq):
    h = F.fqnm_create(F.make_flux("linear_upwind", a=1.0), 2.0 ** -10, 0.01, 0.005)
    with pytest.raises(F.FqnmError) as e:
        F.fqnm_load_states(h, np.zeros(64, dtype=np.int32))
    assert e.value.status == -6
    F.fqnm_destroy(h)
