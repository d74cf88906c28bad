"""The C ABI: the library builds, loads without a GPU and exports every entry point that
include/gks.h declares; host-side validation rejects bad descriptions before any device call."""
import ctypes
import os
import re

import pytest

from paper_2412_16845_gb300 import build as gbuild
from paper_2412_16845_gb300 import gks

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "gks.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gks_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    gbuild.build()
    return gks.load_library()


def test_header_declares_the_step_calls():
    names = declared_functions()
    for must in ("gks_create_mesh", "gks_set_materials", "gks_step", "gks_read_fields"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert names
    for n in names:
        assert hasattr(lib, n), n
    # the binding wraps exactly the declared calls, under the same names
    assert set(gks.SIGNATURES) == set(names)
    for n in names:
        assert callable(getattr(gks, n))


def _desc(**kw):
    d = gks.gks_mesh_desc()
    d.dim, d.kind, d.precision = 2, gks.GKS_CARTESIAN, gks.GKS_FP32
    d.n[0] = d.n[1] = 8
    d.hi[0] = d.hi[1] = 1.0
    d.cfl = 0.5
    for k, v in kw.items():
        setattr(d, k, v)
    return d


@pytest.mark.parametrize("bad", [
    {"dim": 4}, {"precision": 7}, {"cfl": 0.0}, {"cfl": float("nan")}, {"tau_over_dt": -1.0},
    {"kind": 9}, {"chi": -1.0}, {"gamma": float("nan")}, {"limiter": 2}, {"limiter": -1},
])
def test_create_rejects_bad_descriptions(lib, bad):
    d = _desc(**bad)
    ctx = ctypes.c_void_p()
    assert lib.gks_create_mesh(ctypes.byref(d), ctypes.byref(ctx)) == gks.GKS_E_ARG
    assert not ctx.value


def test_create_rejects_unpaired_periodic_and_bad_box(lib):
    d = _desc()
    d.bc[0] = gks.GKS_BC_PERIODIC
    d.bc[1] = gks.GKS_BC_NONREFLECTING
    ctx = ctypes.c_void_p()
    assert lib.gks_create_mesh(ctypes.byref(d), ctypes.byref(ctx)) == gks.GKS_E_ARG
    d = _desc()
    d.hi[0] = -1.0
    assert lib.gks_create_mesh(ctypes.byref(d), ctypes.byref(ctx)) == gks.GKS_E_ARG
    d = _desc()
    d.n[1] = 0
    assert lib.gks_create_mesh(ctypes.byref(d), ctypes.byref(ctx)) == gks.GKS_E_ARG
    assert lib.gks_create_mesh(None, ctypes.byref(ctx)) == gks.GKS_E_ARG
    assert lib.gks_last_error(None) == b"null context"


def test_cleaning_needs_a_cartesian_grid(lib):
    d = _desc(kind=gks.GKS_TET, dim=3, chi=0.5, gamma=0.5)
    ctx = ctypes.c_void_p()
    assert lib.gks_create_mesh(ctypes.byref(d), ctypes.byref(ctx)) == gks.GKS_E_UNSUPPORTED
    assert not ctx.value


def test_limiter_needs_a_cartesian_grid(lib):
    ctx = ctypes.c_void_p()
    d = _desc(kind=gks.GKS_TET, dim=3, limiter=gks.GKS_LIMITER_VAN_LEER)
    assert lib.gks_create_mesh(ctypes.byref(d), ctypes.byref(ctx)) == gks.GKS_E_UNSUPPORTED
    assert not ctx.value
