"""Thin ctypes binding of the C ABI in ``include/gks.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls and does no arithmetic of the
method: all steps run in the CUDA library.  The library is loaded from this package directory
(``libgks.so``, produced by ``paper_2412_16845_gb300.build.build()``); if it is missing, every
call raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgks.so")

GKS_OK, GKS_E_ARG, GKS_E_NOMEM, GKS_E_CUDA, GKS_E_UNSUPPORTED, GKS_E_STATE, \
    GKS_E_NONFINITE, GKS_E_TIMEOUT = range(8)
GKS_CARTESIAN, GKS_TET = 0, 1
GKS_FP32, GKS_FP64 = 0, 1
GKS_BC_PERIODIC, GKS_BC_NONREFLECTING, GKS_BC_PEC = 0, 1, 2
GKS_LIMITER_NONE, GKS_LIMITER_VAN_LEER = 0, 1
_LIMITER = {None: GKS_LIMITER_NONE, "none": GKS_LIMITER_NONE, "vanleer": GKS_LIMITER_VAN_LEER}

STATUS_NAMES = {0: "GKS_OK", 1: "GKS_E_ARG", 2: "GKS_E_NOMEM", 3: "GKS_E_CUDA",
                4: "GKS_E_UNSUPPORTED", 5: "GKS_E_STATE", 6: "GKS_E_NONFINITE",
                7: "GKS_E_TIMEOUT"}


class GksError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


GKS_HALO_OWNED, GKS_HALO_GHOST = 0, 1


class gks_slab_desc(ctypes.Structure):
    _fields_ = [("begin", ctypes.c_int64), ("end", ctypes.c_int64),
                ("shared_lo", ctypes.c_int32), ("shared_hi", ctypes.c_int32)]


class gks_mesh_desc(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32), ("kind", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("reserved0", ctypes.c_int32),
        ("n", ctypes.c_int64 * 3), ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
        ("bc", ctypes.c_int32 * 6),
        ("n_vert", ctypes.c_int64), ("vert_xyz", ctypes.POINTER(ctypes.c_double)),
        ("n_tet", ctypes.c_int64), ("tet_vert", ctypes.POINTER(ctypes.c_int64)),
        ("tet_bc", ctypes.c_int32), ("reserved1", ctypes.c_int32),
        ("cfl", ctypes.c_double), ("tau_over_dt", ctypes.c_double),
        ("c_lattice", ctypes.c_double), ("cuda_stream", ctypes.c_void_p),
        ("chi", ctypes.c_double), ("gamma", ctypes.c_double),
        ("limiter", ctypes.c_int32), ("reserved2", ctypes.c_int32),
    ]


_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)
_CTX = ctypes.c_void_p

# name -> (restype, argtypes)
SIGNATURES = {
    "gks_create_mesh": (ctypes.c_int, [ctypes.POINTER(gks_mesh_desc), ctypes.POINTER(_CTX)]),
    "gks_set_materials": (ctypes.c_int, [_CTX, _D, _D]),
    "gks_write_fields": (ctypes.c_int, [_CTX, _D, ctypes.c_double]),
    "gks_set_source": (ctypes.c_int, [_CTX, _D, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double]),
    "gks_set_source_cw": (ctypes.c_int, [_CTX, _D, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double]),
    "gks_set_materials_box": (ctypes.c_int, [_CTX, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                             ctypes.c_int64, _D]),
    "gks_reset_objective": (ctypes.c_int, [_CTX]),
    "gks_set_dt": (ctypes.c_int, [_CTX, ctypes.c_double]),
    "gks_step": (ctypes.c_int, [_CTX, ctypes.c_int64]),
    "gks_read_fields": (ctypes.c_int, [_CTX, _D]),
    "gks_energy": (ctypes.c_int, [_CTX, _D]),
    "gks_sync": (ctypes.c_int, [_CTX]),
    "gks_set_objective": (ctypes.c_int, [_CTX, _I64, ctypes.c_int64, _I64, ctypes.c_int64]),
    "gks_objective": (ctypes.c_int, [_CTX, _D]),
    "gks_state_layout": (ctypes.c_int, [_CTX, _I64, _I64]),
    "gks_copy_state": (ctypes.c_int, [_CTX, ctypes.c_void_p]),
    "gks_copy_state_box": (ctypes.c_int, [_CTX, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                          ctypes.c_int64, ctypes.c_int64]),
    "gks_step_window": (ctypes.c_int, [_CTX, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                       ctypes.c_int64, ctypes.c_int64]),
    "gks_load_state": (ctypes.c_int, [_CTX, ctypes.c_void_p, ctypes.c_int64]),
    "gks_adjoint_seed": (ctypes.c_int, [_CTX, ctypes.c_void_p, ctypes.c_void_p]),
    "gks_adjoint_step": (ctypes.c_int, [_CTX, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]),
    "gks_energy_noalloc": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                          ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "gks_create_slab": (ctypes.c_int, [ctypes.POINTER(gks_mesh_desc),
                                       ctypes.POINTER(gks_slab_desc), ctypes.POINTER(_CTX)]),
    "gks_halo_bytes": (ctypes.c_int, [_CTX, _I64]),
    "gks_halo_export": (ctypes.c_int, [_CTX, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    "gks_halo_import": (ctypes.c_int, [_CTX, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_int32]),
    "gks_get_info": (ctypes.c_int, [_CTX, _D, _D, _I64, _I64, _D]),
    "gks_get_launch_count": (ctypes.c_int, [_CTX, _I64]),
    "gks_last_error": (ctypes.c_char_p, [_CTX]),
    "gks_destroy": (None, [_CTX]),
}


def load_library(path: str = LIB_PATH):
    """Load ``libgks.so`` (once) and attach the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is not built; run "
                           "paper_2412_16845_gb300.build.build() (there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _dptr(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _check(ctx, status):
    if status != GKS_OK:
        msg = load_library().gks_last_error(ctx)
        raise GksError(status, msg.decode() if msg else "")


def _f64(a, size):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.size != size:
        raise ValueError(f"expected {size} values, got {a.size}")
    return a


# ------------------------------------------------------------------------ same-name wrappers

def gks_create_mesh(desc: gks_mesh_desc):
    ctx = _CTX()
    st = load_library().gks_create_mesh(ctypes.byref(desc), ctypes.byref(ctx))
    if st != GKS_OK:
        raise GksError(st, "gks_create_mesh rejected the description")
    return ctx


def gks_create_slab(desc: gks_mesh_desc, slab: gks_slab_desc):
    ctx = _CTX()
    st = load_library().gks_create_slab(ctypes.byref(desc), ctypes.byref(slab), ctypes.byref(ctx))
    if st != GKS_OK:
        raise GksError(st, "gks_create_slab rejected the description")
    return ctx


def gks_halo_bytes(ctx):
    v = ctypes.c_int64()
    _check(ctx, load_library().gks_halo_bytes(ctx, ctypes.byref(v)))
    return v.value


def gks_halo_export(ctx, side, layers, state_ptr, buf_ptr):
    _check(ctx, load_library().gks_halo_export(ctx, int(side), int(layers), state_ptr or None,
                                               buf_ptr))


def gks_halo_import(ctx, side, layers, state_ptr, buf_ptr, add=False):
    _check(ctx, load_library().gks_halo_import(ctx, int(side), int(layers), state_ptr or None,
                                               buf_ptr, 1 if add else 0))


def gks_set_materials(ctx, eps, mu=None):
    _check(ctx, load_library().gks_set_materials(ctx, _dptr(eps), _dptr(mu)))


def gks_write_fields(ctx, fields, t0=0.0):
    _check(ctx, load_library().gks_write_fields(ctx, _dptr(fields), float(t0)))


def gks_set_source(ctx, jz_mask, A, f0, t0, s):
    _check(ctx, load_library().gks_set_source(ctx, _dptr(jz_mask), A, f0, t0, s))


def gks_set_source_cw(ctx, jz_mask, A, f0, t0):
    _check(ctx, load_library().gks_set_source_cw(ctx, _dptr(jz_mask), A, f0, t0))


def gks_set_materials_box(ctx, x0, x1, y0, y1, eps_box):
    eps_box = np.ascontiguousarray(eps_box, dtype=np.float64)
    if eps_box.size != (x1 - x0) * (y1 - y0):
        raise ValueError("eps_box must hold (y1 - y0) * (x1 - x0) values")
    _check(ctx, load_library().gks_set_materials_box(ctx, int(x0), int(x1), int(y0), int(y1),
                                                     eps_box.ctypes.data_as(_D)))


def gks_reset_objective(ctx):
    _check(ctx, load_library().gks_reset_objective(ctx))


def gks_set_dt(ctx, dt):
    _check(ctx, load_library().gks_set_dt(ctx, float(dt)))


def gks_step(ctx, n_steps):
    _check(ctx, load_library().gks_step(ctx, int(n_steps)))


def gks_read_fields(ctx, out):
    _check(ctx, load_library().gks_read_fields(ctx, _dptr(out)))
    return out


def gks_energy(ctx):
    v = ctypes.c_double()
    _check(ctx, load_library().gks_energy(ctx, ctypes.byref(v)))
    return v.value


def gks_energy_noalloc(precision, dim, n_cells, cell_volume, fields_ptr, eps_ptr, mu_ptr,
                       out_ptr, stream=0):
    """Energy of caller-owned device arrays (device pointers as ints) into the device double at
    out_ptr; no allocation.  Raises GksError on a non-OK status."""
    st = load_library().gks_energy_noalloc(int(precision), int(dim), int(n_cells),
                                           float(cell_volume), fields_ptr, eps_ptr, mu_ptr,
                                           out_ptr, stream or None)
    if st != GKS_OK:
        raise GksError(st, "gks_energy_noalloc rejected the call")


def gks_set_objective(ctx, probe, design):
    probe = np.ascontiguousarray(probe if probe is not None else [], dtype=np.int64)
    design = np.ascontiguousarray(design if design is not None else [], dtype=np.int64)
    _check(ctx, load_library().gks_set_objective(ctx, probe.ctypes.data_as(_I64), probe.size,
                                                 design.ctypes.data_as(_I64), design.size))


def gks_objective(ctx):
    v = ctypes.c_double()
    _check(ctx, load_library().gks_objective(ctx, ctypes.byref(v)))
    return v.value


def gks_state_layout(ctx):
    n, b = ctypes.c_int64(), ctypes.c_int64()
    _check(ctx, load_library().gks_state_layout(ctx, ctypes.byref(n), ctypes.byref(b)))
    return n.value, b.value


def gks_copy_state(ctx, dst_ptr):
    _check(ctx, load_library().gks_copy_state(ctx, dst_ptr))


def gks_copy_state_box(ctx, dst_ptr, x0, x1, y0, y1):
    _check(ctx, load_library().gks_copy_state_box(ctx, dst_ptr, int(x0), int(x1), int(y0), int(y1)))


def gks_step_window(ctx, n_steps, x0, x1, y0, y1):
    _check(ctx, load_library().gks_step_window(ctx, int(n_steps), int(x0), int(x1), int(y0),
                                               int(y1)))


def gks_load_state(ctx, src_ptr, step):
    _check(ctx, load_library().gks_load_state(ctx, src_ptr, int(step)))


def gks_adjoint_seed(ctx, state_ptr, adj_ptr):
    _check(ctx, load_library().gks_adjoint_seed(ctx, state_ptr, adj_ptr))


def gks_adjoint_step(ctx, state_n, state_np1, adj_in, adj_out, grad_eps, add_probe):
    _check(ctx, load_library().gks_adjoint_step(ctx, state_n, state_np1, adj_in, adj_out,
                                                grad_eps, 1 if add_probe else 0))


def gks_sync(ctx):
    _check(ctx, load_library().gks_sync(ctx))


def gks_get_info(ctx):
    dt, t, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    step, n = ctypes.c_int64(), ctypes.c_int64()
    _check(ctx, load_library().gks_get_info(ctx, ctypes.byref(dt), ctypes.byref(t),
                                            ctypes.byref(step), ctypes.byref(n),
                                            ctypes.byref(c)))
    return {"dt": dt.value, "t": t.value, "step": step.value, "n_cells": n.value,
            "c": c.value}


def gks_get_launch_count(ctx):
    n = ctypes.c_int64()
    _check(ctx, load_library().gks_get_launch_count(ctx, ctypes.byref(n)))
    return n.value


def gks_last_error(ctx):
    msg = load_library().gks_last_error(ctx)
    return msg.decode() if msg else ""


def gks_destroy(ctx):
    load_library().gks_destroy(ctx)


# ------------------------------------------------------------------------ convenience class

_BC = {"periodic": GKS_BC_PERIODIC, "nrbc": GKS_BC_NONREFLECTING, "pec": GKS_BC_PEC}


@dataclass
class SolverSpec:
    dim: int
    n: tuple
    lo: tuple
    hi: tuple
    bc: tuple
    cfl: float
    precision: str = "fp32"
    kappa: float = 0.0
    c_lattice: float = 0.0
    phm: tuple | None = None          # (chi, gamma) divergence cleaning (Cartesian grids)
    limiter: str | None = None        # None or "vanleer" (Cartesian grids)


class GKSSolver:
    """One GKS context (owning its device state) with numpy in/out in user order."""

    def __init__(self, spec: SolverSpec, stream: int = 0):
        d = gks_mesh_desc()
        d.dim = spec.dim
        d.kind = GKS_CARTESIAN
        d.precision = GKS_FP64 if spec.precision == "fp64" else GKS_FP32
        for a in range(spec.dim):
            d.n[a] = int(spec.n[a])
            d.lo[a] = float(spec.lo[a])
            d.hi[a] = float(spec.hi[a])
        for s, b in enumerate(spec.bc):
            d.bc[s] = _BC[b] if isinstance(b, str) else int(b)
        d.cfl = spec.cfl
        d.tau_over_dt = spec.kappa
        d.c_lattice = spec.c_lattice
        d.cuda_stream = ctypes.c_void_p(int(stream)) if stream else None
        cleaning = spec.phm is not None and (spec.phm[0] > 0 or spec.phm[1] > 0)
        if spec.phm is not None:
            d.chi, d.gamma = float(spec.phm[0]), float(spec.phm[1])
        d.limiter = _LIMITER[spec.limiter]
        self.spec = spec
        self.ncomp = (4 if cleaning else 3) if spec.dim == 2 else (8 if cleaning else 6)
        self.ncell = int(np.prod(spec.n[: spec.dim]))
        self.ctx = gks_create_mesh(d)

    @classmethod
    def from_tets(cls, vert, tet, cfl, precision="fp32", kappa=0.0, c_lattice=1.0, stream=0,
                  bc="nrbc"):
        """A context on a conforming tetrahedral mesh (vert [nv][3], tet [nt][4]); every boundary
        face is kinetic non-reflecting (bc="nrbc") or a PEC wall (bc="pec")."""
        vert = np.ascontiguousarray(vert, dtype=np.float64)
        tet = np.ascontiguousarray(tet, dtype=np.int64)
        d = gks_mesh_desc()
        d.dim = 3
        d.kind = GKS_TET
        d.precision = GKS_FP64 if precision == "fp64" else GKS_FP32
        d.n_vert = vert.shape[0]
        d.vert_xyz = vert.ctypes.data_as(_D)
        d.n_tet = tet.shape[0]
        d.tet_vert = tet.ctypes.data_as(_I64)
        d.tet_bc = _BC[bc]
        d.cfl = cfl
        d.tau_over_dt = kappa
        d.c_lattice = c_lattice
        d.cuda_stream = ctypes.c_void_p(int(stream)) if stream else None
        self = cls.__new__(cls)
        self.spec = None
        self.ncomp = 6
        self.ncell = int(tet.shape[0])
        self.ctx = gks_create_mesh(d)
        return self

    @classmethod
    def from_tet_workload(cls, w, precision="fp32", kappa=0.0, stream=0):
        s = cls.from_tets(w.vert, w.tet, w.cfl, precision=precision, kappa=kappa, stream=stream)
        s.set_materials(w.eps, w.mu)
        s.write_fields(w.fields0)
        return s

    @classmethod
    def from_workload(cls, w, precision="fp32", kappa=0.0, stream=0, c_lattice=None):
        """c_lattice: the lattice speed c; None takes the workload's (0 = fastest wave)."""
        if c_lattice is None:
            c_lattice = getattr(w, "c_lattice", 0.0) or 0.0
        s = cls(SolverSpec(dim=w.dim, n=w.n, lo=w.lo, hi=w.hi, bc=w.bc, cfl=w.cfl,
                           precision=precision, kappa=kappa, c_lattice=c_lattice,
                           phm=getattr(w, "phm", None),
                           limiter=getattr(w, "limiter", None)), stream=stream)
        s.set_materials(w.eps, w.mu)
        s.write_fields(w.fields0)
        if w.jz_mask is not None:
            if getattr(w, "waveform", "gauss_sine") == "cw":
                s.set_source_cw(w.jz_mask, *w.src)
            else:
                s.set_source(w.jz_mask, *w.src)
        return s

    def set_materials(self, eps, mu=None):
        eps = _f64(eps, self.ncell)
        mu = None if mu is None else _f64(mu, self.ncell)
        gks_set_materials(self.ctx, eps, mu)

    def write_fields(self, fields, t0=0.0):
        """fields [ncomp][n_cells]; with divergence cleaning the potentials may be left out
        (the electromagnetic rows alone), and then start at zero."""
        f = np.asarray(fields, dtype=np.float64)
        base = 3 if self.spec is not None and self.spec.dim == 2 else 6
        if self.ncomp > base and f.size == base * self.ncell:
            f = np.concatenate([f.reshape(base, self.ncell),
                                np.zeros((self.ncomp - base, self.ncell))])
        gks_write_fields(self.ctx, _f64(f, self.ncomp * self.ncell), t0)

    def set_source(self, jz_mask, A, f0, t0, s):
        gks_set_source(self.ctx, None if jz_mask is None else _f64(jz_mask, self.ncell),
                       A, f0, t0, s)

    def set_source_cw(self, jz_mask, A, f0, t0=0.0):
        gks_set_source_cw(self.ctx, None if jz_mask is None else _f64(jz_mask, self.ncell),
                          A, f0, t0)

    def set_dt(self, dt):
        gks_set_dt(self.ctx, dt)

    def step(self, n=1):
        gks_step(self.ctx, n)

    def read_fields(self, out=None):
        if out is None:
            out = np.empty((self.ncomp, self.ncell), dtype=np.float64)
        return gks_read_fields(self.ctx, out)

    def energy(self):
        return gks_energy(self.ctx)

    def sync(self):
        gks_sync(self.ctx)

    def info(self):
        return gks_get_info(self.ctx)

    def launch_count(self):
        return gks_get_launch_count(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            gks_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
