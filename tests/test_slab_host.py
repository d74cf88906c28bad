"""The domain split across ranks (paper_2412_16845_gb300/slab.py) on CPU ranks over gloo.

Each rank holds a slab of the slowest axis plus two ghost layers per shared side and advances
it with the FP64 oracle on its local grid (standing in for the CUDA library, which needs a GPU;
the GPU version of the same exchange is in test_gpu_slab.py).  After every step the ranks swap
their boundary layers with ``slab.exchange`` through torch.distributed point-to-point calls.
The owned cells then equal the oracle run on the whole grid (the update of Sec. 3.1 has a
two-cell reach, so two ghost layers suffice), for 2-D and 3-D grids, periodic and
non-reflecting slab axes, 2 and 3 ranks.  The energies summed in rank order equal the whole
grid's.  The transposed exchange (ghost layers added into the neighbour's owned layers) is the
adjoint of the forward copy: <P x, y> = <x, P^T y> over all ranks."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_partition_covers_the_axis():
    from paper_2412_16845_gb300.slab import partition
    for n, world, periodic in ((10, 3, False), (7, 2, True), (8, 4, False), (5, 1, True)):
        plans = [partition(n, world, r, periodic) for r in range(world)]
        owned = np.concatenate([np.arange(p.begin, p.end) for p in plans])
        assert np.array_equal(owned, np.arange(n))
        sizes = [p.end - p.begin for p in plans]
        assert max(sizes) - min(sizes) <= 1
        for p in plans:
            if world == 1:
                assert not p.shared_lo and not p.shared_hi and p.n_local == n
                continue
            if periodic:
                assert p.shared_lo and p.shared_hi
                assert p.rank_lo == (p.rank - 1) % world and p.rank_hi == (p.rank + 1) % world
            else:
                assert p.shared_lo == (p.rank > 0) and p.shared_hi == (p.rank < world - 1)
            gl = p.global_layers()
            assert gl.size == p.n_local and np.all(gl[p.own0:p.own0 + p.end - p.begin] ==
                                                   np.arange(p.begin, p.end))
    with pytest.raises(ValueError):
        partition(5, 3, 0, False)          # a rank would own fewer than two layers


def _case(dim, periodic_axis, seed):
    """A small workload with random fields and eps."""
    from paper_2412_16845_gb300 import workloads as wl
    rng = np.random.default_rng(seed)
    n = (7, 13) if dim == 2 else (5, 4, 11)
    h = 0.1
    ncell = int(np.prod(n))
    bc = ["nrbc"] * (2 * dim)
    bc[2 * dim - 2] = bc[2 * dim - 1] = "periodic" if periodic_axis else "nrbc"
    ncomp = 3 if dim == 2 else 6
    return wl.CartWorkload(name="slab", dim=dim, n=n, lo=(0.0,) * dim,
                           hi=tuple(h * v for v in n), bc=tuple(bc), cfl=0.4, steps=0,
                           eps=rng.uniform(1.0, 3.0, ncell), mu=None,
                           fields0=rng.standard_normal((ncomp, ncell)), c_lattice=1.0)


def _rank_main(rank, world, port, dim, periodic_axis, nsteps, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from oracle import gks_oracle as go
    from paper_2412_16845_gb300 import slab
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = _case(dim, periodic_axis, 5)
        ax = dim - 1
        plan = slab.partition(w.n[ax], world, rank, periodic_axis)
        cpl = int(np.prod(w.n[:ax]))
        ids = slab.local_cells(plan, cpl)
        # the whole grid's dt; the local grid with non-reflecting edges at shared sides
        whole = go.cartesian_mesh(w.n, w.lo, w.hi, w.bc)
        dt = go.time_step(whole, w.cfl)
        C = go.time_coefficients(dt, 0.0)
        h = (w.hi[ax] - w.lo[ax]) / w.n[ax]
        lo, hi, bc = list(w.lo), list(w.hi), list(w.bc)
        lo[ax] = w.lo[ax] + plan.first * h
        hi[ax] = lo[ax] + plan.n_local * h
        if plan.shared_lo or plan.shared_hi:
            bc[2 * ax] = "nrbc" if plan.shared_lo else bc[2 * ax]
            bc[2 * ax + 1] = "nrbc" if plan.shared_hi else bc[2 * ax + 1]
        n_loc = list(w.n)
        n_loc[ax] = plan.n_local
        mesh = go.cartesian_mesh(tuple(n_loc), tuple(lo), tuple(hi), tuple(bc))
        V = go.fields_to_state(w.fields0[:, ids], dim)
        m = go.material_diag(w.eps[ids], None)
        o0 = plan.own0 * cpl
        o1 = (plan.own0 + plan.end - plan.begin) * cpl

        def rows(side, layers):
            if layers == "owned":
                a = o0 if side == 0 else o1 - 2 * cpl
            else:
                a = o0 - 2 * cpl if side == 0 else o1
            return slice(a, a + 2 * cpl)

        state = {"V": V}
        nb = 2 * cpl * V.shape[1]
        send = [torch.zeros(nb, dtype=torch.float64) for _ in range(2)]
        recv = [torch.zeros(nb, dtype=torch.float64) for _ in range(2)]

        def export(side, buf):
            buf.copy_(torch.from_numpy(np.ascontiguousarray(state["V"][rows(side, "owned")]).ravel()))

        def import_(side, buf):
            state["V"][rows(side, "ghost")] = buf.numpy().reshape(2 * cpl, -1)

        for _ in range(nsteps):
            state["V"] = go.step(mesh, state["V"], m, dt, C)
            slab.exchange(plan, export, import_, send, recv)
        owned_ids = ids[o0:o1]
        e_local = 0.5 * float(np.sum(mesh.vol[o0:o1, None] * m[o0:o1] * state["V"][o0:o1] ** 2))
        e_total = slab.ordered_sum(e_local)
        # the transposed exchange: <P x, y> = <x, P^T y> summed over ranks
        rng = np.random.default_rng(100 + rank)
        x = rng.standard_normal(state["V"].shape)
        y = rng.standard_normal(state["V"].shape)
        Px = x.copy()
        st = {"V": Px}

        def exp_f(side, buf):
            buf.copy_(torch.from_numpy(np.ascontiguousarray(st["V"][rows(side, "owned")]).ravel()))

        def imp_f(side, buf):
            st["V"][rows(side, "ghost")] = buf.numpy().reshape(2 * cpl, -1)

        slab.exchange(plan, exp_f, imp_f, send, recv)
        # P x: owned part of x kept, ghosts replaced by the neighbours' owned layers; P^T y:
        # ghosts of y sent back and added into the neighbours' owned layers, ghosts dropped
        PTy = y.copy()
        st2 = {"V": PTy}

        def exp_t(side, buf):
            buf.copy_(torch.from_numpy(np.ascontiguousarray(st2["V"][rows(side, "ghost")]).ravel()))

        def imp_t(side, buf):
            st2["V"][rows(side, "owned")] += buf.numpy().reshape(2 * cpl, -1)

        slab.exchange(plan, exp_t, imp_t, send, recv)
        # <P x, y> over every rank's local grid equals <x, P^T y> over the owned cells
        lhs = slab.ordered_sum(float(np.sum(Px * y)))
        rhs = slab.ordered_sum(float(np.sum(x[o0:o1] * PTy[o0:o1])))
        out.put((rank, owned_ids, go.state_to_fields(state["V"][o0:o1], dim), e_total, lhs, rhs))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("dim,periodic_axis,world", [
    (2, False, 2), (2, True, 2), (2, False, 3), (3, False, 2), (3, True, 3),
])
def test_gloo_slabs_match_the_whole_grid(dim, periodic_axis, world):
    import torch.multiprocessing as mp
    from oracle import gks_oracle as go
    nsteps = 5
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, dim, periodic_axis, nsteps, q))
             for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(world)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    w = _case(dim, periodic_axis, 5)
    whole = go.cartesian_mesh(w.n, w.lo, w.hi, w.bc)
    ref, _ = go.run(whole, w.fields0, w.eps, None, w.cfl, nsteps, c=1.0)
    got = np.zeros_like(ref)
    seen = np.zeros(ref.shape[1], dtype=int)
    for _, ids, f, _, _, _ in res:
        got[:, ids] = f
        seen[ids] += 1
    assert np.all(seen == 1)                      # every cell owned by exactly one rank
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    m = go.material_diag(w.eps, None)
    e_ref = go.energy(whole, go.fields_to_state(ref, dim), m)
    for _, _, _, e_total, lhs, rhs in res:
        assert abs(e_total - e_ref) <= 1e-13 * e_ref
        assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))
    # every rank reports the same sums, bit for bit (fixed rank order)
    assert len({r[3] for r in res}) == 1 and len({r[4] for r in res}) == 1
