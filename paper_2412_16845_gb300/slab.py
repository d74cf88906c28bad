"""A Cartesian grid split across ranks: slabs of the slowest axis, two ghost layers per shared
side, a halo exchange after every step (host logic; the library does the device work).

The finite-volume update of Sec. 3.1 reaches two cells along every axis (Green-Gauss gradient,
then the face flux between two reconstructed cells), so each rank advances its slab exactly like
the whole grid once its ghost layers hold the neighbours' owned layers of the same time level.
The slab axis is y in 2-D and z in 3-D (the slowest in the state layout, so a layer is
contiguous).  Ranks exchange their boundary layers point to point after each step; energies are
combined in a fixed rank order.  The transpose of the ghost copy (for adjoint fields) adds the
neighbour's ghost layers into the owned ones: the same ``exchange`` with other callbacks.

Nothing here computes any of the method's arithmetic; the CUDA library steps each slab
(``gks_create_slab``, ``gks_halo_export``, ``gks_halo_import``) and torch.distributed moves the
buffers (NCCL between GPUs, gloo through host memory).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

GHOST = 2          # ghost layers per shared side: the stencil radius of the step


@dataclass(frozen=True)
class SlabPlan:
    rank: int
    world: int
    n_axis: int          # cells of the whole grid along the slab axis
    periodic: bool
    begin: int           # owned cells [begin, end)
    end: int
    shared_lo: bool
    shared_hi: bool
    rank_lo: int         # neighbour across the low side (-1: none)
    rank_hi: int

    @property
    def first(self) -> int:
        """Global index (unwrapped) of the local grid's first layer."""
        return self.begin - GHOST * int(self.shared_lo)

    @property
    def n_local(self) -> int:
        return self.end - self.begin + GHOST * (int(self.shared_lo) + int(self.shared_hi))

    @property
    def own0(self) -> int:
        """Local index of the first owned layer."""
        return GHOST * int(self.shared_lo)

    def global_layers(self) -> np.ndarray:
        """Global layer index of every local layer (wrapped on a periodic axis)."""
        idx = np.arange(self.first, self.first + self.n_local)
        return np.mod(idx, self.n_axis) if self.periodic else idx


def partition(n_axis: int, world: int, rank: int, periodic: bool) -> SlabPlan:
    """Rank ``rank``'s slab of ``n_axis`` layers split as evenly as possible over ``world``
    ranks (the first n_axis % world ranks take one layer more).  Every rank of a split grid owns
    at least two layers, the depth of a neighbour's ghost layers."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    if world > 1 and n_axis < GHOST * world:
        raise ValueError(f"{n_axis} layers cannot give {world} ranks {GHOST} layers each")
    base, extra = divmod(n_axis, world)
    begin = rank * base + min(rank, extra)
    end = begin + base + (1 if rank < extra else 0)
    if world == 1:
        return SlabPlan(rank, world, n_axis, periodic, 0, n_axis, False, False, -1, -1)
    if periodic:
        return SlabPlan(rank, world, n_axis, True, begin, end, True, True,
                        (rank - 1) % world, (rank + 1) % world)
    return SlabPlan(rank, world, n_axis, False, begin, end, rank > 0, rank < world - 1,
                    rank - 1 if rank > 0 else -1, rank + 1 if rank < world - 1 else -1)


def layer_cells(shape_xy: int, layers: np.ndarray) -> np.ndarray:
    """User-order cell ids of the given layers of the slab axis, in local order (x fastest;
    shape_xy = cells per layer)."""
    return (layers[:, None] * shape_xy + np.arange(shape_xy)[None, :]).ravel()


def local_cells(plan: SlabPlan, cells_per_layer: int) -> np.ndarray:
    """Global user-order ids of the local grid's cells (ghost layers included), local order."""
    return layer_cells(cells_per_layer, plan.global_layers())


def owned_local(plan: SlabPlan, cells_per_layer: int) -> np.ndarray:
    """Local user-order ids of the owned cells."""
    return layer_cells(cells_per_layer, np.arange(plan.own0, plan.own0 + plan.end - plan.begin))


def slab_descriptor(plan: SlabPlan):
    from .gks import gks_slab_desc
    d = gks_slab_desc()
    d.begin, d.end = plan.begin, plan.end
    d.shared_lo, d.shared_hi = int(plan.shared_lo), int(plan.shared_hi)
    return d


# ------------------------------------------------------------------------------ exchange
def exchange(plan: SlabPlan, export, import_, send_bufs, recv_bufs):
    """One halo exchange with the neighbours through torch.distributed point-to-point calls.

    export(side, buf) fills buf with this rank's layers for the neighbour across ``side``
    (0 = low, 1 = high); import_(side, buf) takes the neighbour's layers.  The forward step's
    exchange sends owned layers and writes them into the neighbour's ghost layers; its
    transpose, for adjoint fields, sends ghost layers and adds them into the neighbour's owned
    layers (the callbacks choose).  send_bufs / recv_bufs: per side, tensors on the backend's
    device (CUDA for NCCL, CPU for gloo) that export/import use.

    A rank's high side pairs with the next rank's low side.  Sends go out high side first and
    receives are posted low side first, so that two ranks of a ring, neighbours across both
    sides, match their messages in order (tags say the same for backends that use them)."""
    import torch.distributed as dist

    sides = [s for s in (0, 1) if (plan.shared_lo if s == 0 else plan.shared_hi)]
    if not sides:
        return
    peer = {0: plan.rank_lo, 1: plan.rank_hi}
    for s in sides:
        export(s, send_bufs[s])
    ops = []
    for s in sorted(sides, reverse=True):
        ops.append(dist.P2POp(dist.isend, send_bufs[s], peer[s], tag=1 - s))
    for s in sides:
        ops.append(dist.P2POp(dist.irecv, recv_bufs[s], peer[s], tag=s))
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    for s in sides:
        import_(s, recv_bufs[s])


def ordered_sum(value: float) -> float:
    """Sum of one FP64 value per rank, added in rank order on every rank (deterministic)."""
    import torch
    import torch.distributed as dist

    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    dev = torch.device("cuda", torch.cuda.current_device()) \
        if dist.get_backend() == "nccl" else torch.device("cpu")
    mine = torch.tensor([value], dtype=torch.float64, device=dev)
    parts = [torch.zeros_like(mine) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, mine)
    total = 0.0
    for p in parts:
        total += float(p.item())
    return total


# ------------------------------------------------------------------------------ one rank
class SlabSolver:
    """One rank's slab of a Cartesian workload (``workloads.CartWorkload``), stepped by the CUDA
    library, with its halo buffers.  ``backend`` is the torch.distributed backend the
    exchange runs over: "nccl" moves device buffers, "gloo" stages them through host memory.
    The lattice speed is fixed for all ranks: the workload's, else the fastest wave of the
    whole grid's materials."""

    def __init__(self, w, plan: SlabPlan, precision="fp32", kappa=0.0, backend="nccl",
                 stream=None):
        import ctypes

        import torch

        from . import gks as G

        self.w, self.plan, self.backend = w, plan, backend
        c = getattr(w, "c_lattice", 0.0) or 0.0
        if c <= 0.0:
            mu = np.ones_like(w.eps) if w.mu is None else w.mu
            c = max(1.0, float(np.max(1.0 / np.sqrt(np.asarray(w.eps) * mu))))
        self.c = c
        d = G.gks_mesh_desc()
        d.dim, d.kind = w.dim, G.GKS_CARTESIAN
        d.precision = G.GKS_FP64 if precision == "fp64" else G.GKS_FP32
        for a in range(w.dim):
            d.n[a], d.lo[a], d.hi[a] = int(w.n[a]), float(w.lo[a]), float(w.hi[a])
        for k, b in enumerate(w.bc):
            d.bc[k] = G._BC[b]
        d.cfl, d.tau_over_dt, d.c_lattice = w.cfl, kappa, c
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        d.cuda_stream = ctypes.c_void_p(int(stream)) if stream else None
        if getattr(w, "phm", None) is not None:
            d.chi, d.gamma = float(w.phm[0]), float(w.phm[1])
        d.limiter = G._LIMITER[getattr(w, "limiter", None)]
        self.ctx = G.gks_create_slab(d, slab_descriptor(plan))
        self.cells_per_layer = int(np.prod(w.n[: w.dim - 1]))
        self.ids = local_cells(plan, self.cells_per_layer)
        self.owned = owned_local(plan, self.cells_per_layer)
        self.ncell = self.ids.size
        self.ncomp = np.asarray(w.fields0).shape[0]
        G.gks_set_materials(self.ctx, np.ascontiguousarray(np.asarray(w.eps)[self.ids]),
                            None if w.mu is None else np.ascontiguousarray(np.asarray(w.mu)[self.ids]))
        G.gks_write_fields(self.ctx, np.ascontiguousarray(np.asarray(w.fields0)[:, self.ids]))
        if w.jz_mask is not None:
            m = np.ascontiguousarray(np.asarray(w.jz_mask)[self.ids])
            if getattr(w, "waveform", "gauss_sine") == "cw":
                G.gks_set_source_cw(self.ctx, m, *w.src)
            else:
                G.gks_set_source(self.ctx, m, *w.src)
        nbytes = G.gks_halo_bytes(self.ctx) if (plan.shared_lo or plan.shared_hi) else 0
        dev = torch.device("cuda", torch.cuda.current_device())
        self.dev_send = [torch.empty(nbytes, dtype=torch.uint8, device=dev) for _ in range(2)]
        self.dev_recv = [torch.empty(nbytes, dtype=torch.uint8, device=dev) for _ in range(2)]
        if backend == "nccl":
            self.send, self.recv = self.dev_send, self.dev_recv
        else:
            self.send = [torch.empty(nbytes, dtype=torch.uint8).pin_memory() if nbytes else
                         torch.empty(0, dtype=torch.uint8) for _ in range(2)]
            self.recv = [torch.empty_like(b) for b in self.send]

    # callbacks of the forward exchange (owned layers out, ghost layers in)
    def _export(self, side, buf):
        from . import gks as G
        G.gks_halo_export(self.ctx, side, G.GKS_HALO_OWNED, None, self.dev_send[side].data_ptr())
        if buf is not self.dev_send[side]:
            buf.copy_(self.dev_send[side])

    def _import(self, side, buf):
        from . import gks as G
        if buf is not self.dev_recv[side]:
            self.dev_recv[side].copy_(buf)
        G.gks_halo_import(self.ctx, side, G.GKS_HALO_GHOST, None, self.dev_recv[side].data_ptr(),
                          False)

    def exchange(self):
        exchange(self.plan, self._export, self._import, self.send, self.recv)

    def step(self, n=1):
        from . import gks as G
        for _ in range(int(n)):
            G.gks_step(self.ctx, 1)
            self.exchange()

    def read_owned(self):
        """The owned cells' fields [ncomp][owned], ordered like their global ids
        (``self.ids[self.owned]``)."""
        from . import gks as G
        out = np.empty((self.ncomp, self.ncell))
        G.gks_read_fields(self.ctx, out)
        return out[:, self.owned]

    def energy(self):
        """Energy of the whole grid: each rank's owned cells, summed in rank order."""
        from . import gks as G
        return ordered_sum(G.gks_energy(self.ctx))

    def info(self):
        from . import gks as G
        return G.gks_get_info(self.ctx)

    def close(self):
        from . import gks as G
        if getattr(self, "ctx", None):
            G.gks_destroy(self.ctx)
            self.ctx = None
