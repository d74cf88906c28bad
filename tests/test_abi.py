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


def _tet_desc(vert, tet, tet_bc=None):
    """A tet-mesh description over host arrays (kept alive by the caller)."""
    d = _desc(kind=gks.GKS_TET, dim=3)
    d.n_vert = vert.shape[0]
    d.vert_xyz = vert.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d.n_tet = tet.shape[0]
    d.tet_vert = tet.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    d.tet_bc = gks.GKS_BC_NONREFLECTING if tet_bc is None else tet_bc
    return d


@pytest.mark.parametrize("case", ["vertex_id", "non_finite", "degenerate", "three_owners",
                                  "wall_kind"])
def test_create_rejects_bad_tet_meshes(lib, case):
    """The host builds the FP64 geometry before any device memory exists, and rejects a mesh
    whose vertex ids leave the vertex list, whose coordinates are not finite, with a tet of zero
    volume, with a face of three tets, or with an unknown wall kind."""
    import numpy as np
    vert = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [0, 0, -1], [1, 1, 1]], float)
    tet = np.array([[0, 1, 2, 3], [0, 1, 2, 4]], np.int64)
    bc = None
    if case == "vertex_id":
        tet[1, 3] = 6
    elif case == "non_finite":
        vert[5, 0] = np.inf
    elif case == "degenerate":
        vert[4] = [0.5, 0.5, 0.0]                   # in the plane of face (0, 1, 2)
    elif case == "three_owners":
        tet = np.array([[0, 1, 2, 3], [0, 1, 2, 4], [0, 1, 2, 5]], np.int64)
    else:
        bc = gks.GKS_BC_PERIODIC
    d = _tet_desc(vert, tet, bc)
    ctx = ctypes.c_void_p()
    assert lib.gks_create_mesh(ctypes.byref(d), ctypes.byref(ctx)) == gks.GKS_E_ARG
    assert not ctx.value


@pytest.mark.parametrize("args", [
    (7, 2, 10, 1.0), (gks.GKS_FP32, 4, 10, 1.0), (gks.GKS_FP32, 2, 0, 1.0),
    (gks.GKS_FP32, 2, 33554432 + 1, 1.0), (gks.GKS_FP64, 3, 10, 0.0),
    (gks.GKS_FP64, 3, 10, float("nan")),
])
def test_noalloc_energy_rejects_bad_arguments(lib, args):
    """gks_energy_noalloc checks its precision, dimension, cell count (at most the fixed scratch's
    33,554,432 cells) and cell volume before it touches the device."""
    precision, dim, n, vol = args
    fake = ctypes.c_void_p(256)                     # never dereferenced: rejected first
    out = ctypes.c_void_p(512)
    assert lib.gks_energy_noalloc(precision, dim, ctypes.c_int64(n), ctypes.c_double(vol), fake,
                                  fake, None, out, None) == gks.GKS_E_ARG


@pytest.mark.parametrize("case", ["auto_speed", "flag", "empty", "past_end", "thin", "ring",
                                  "edge", "tets"])
def test_create_slab_rejects_bad_slabs(lib, case):
    """A rank-local slab needs the whole grid's lattice speed, 0/1 sharing flags, a non-empty
    range inside the grid, two owned layers for each neighbour, both sides shared on a periodic
    axis, no shared side at a non-periodic grid edge, and a Cartesian grid."""
    d = _desc(c_lattice=1.0)                         # 8 x 8; slab axis y
    d.bc[2] = d.bc[3] = gks.GKS_BC_NONREFLECTING     # (the zero-filled sides are periodic)
    s = gks.gks_slab_desc(begin=2, end=6, shared_lo=1, shared_hi=1)
    if case == "auto_speed":
        d.c_lattice = 0.0
    elif case == "flag":
        s.shared_hi = 2
    elif case == "empty":
        s.end = 2
    elif case == "past_end":
        s.end = 9
    elif case == "thin":
        s.end = 3
    elif case == "ring":
        d.bc[2] = d.bc[3] = gks.GKS_BC_PERIODIC
        s.shared_hi = 0
    elif case == "edge":
        s.begin = 0
    else:
        d.kind = gks.GKS_TET
    ctx = ctypes.c_void_p()
    assert lib.gks_create_slab(ctypes.byref(d), ctypes.byref(s), ctypes.byref(ctx)) == \
        gks.GKS_E_ARG
    assert not ctx.value
