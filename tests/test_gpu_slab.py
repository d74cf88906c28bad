"""A grid split into slabs (gks_create_slab, gks_halo_export, gks_halo_import) on one GPU: two or
three rank contexts in one process, their boundary layers exchanged through host memory after
every step, against the FP64 oracle on the whole grid (relative L2 <= 1e-12 in FP64, <= 2e-5 in
FP32); the owned energies sum to the whole grid's; the library's transposed exchange (ghost
layers added into the neighbour's owned layers) is the adjoint of its forward copy."""
import numpy as np
import pytest

from oracle import gks_oracle as go
from paper_2412_16845_gb300 import gks as G
from paper_2412_16845_gb300 import slab
from paper_2412_16845_gb300 import workloads as wl
from tests.oracle_runs import rel_l2

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2412_16845_gb300 import build
    build.build()


def _case(dim, periodic_axis, seed, with_src):
    rng = np.random.default_rng(seed)
    n = (37, 29) if dim == 2 else (20, 9, 17)
    h = 1.0 / n[0]
    ncell = int(np.prod(n))
    bc = ["nrbc"] * (2 * dim)
    bc[2 * dim - 2] = bc[2 * dim - 1] = "periodic" if periodic_axis else "nrbc"
    ncomp = 3 if dim == 2 else 6
    mask = None
    if with_src:
        mask = np.zeros(ncell)
        mask[rng.choice(ncell, size=6, replace=False)] = rng.uniform(-2, 2, 6)
    return wl.CartWorkload(name="slab", dim=dim, n=n, lo=(0.0,) * dim,
                           hi=tuple(h * v for v in n), bc=tuple(bc), cfl=0.4, steps=0,
                           eps=rng.uniform(1.0, 3.0, ncell), mu=None,
                           fields0=rng.standard_normal((ncomp, ncell)), jz_mask=mask,
                           src=(1.0, 20.0, 0.02, 0.02), c_lattice=1.0)


def _exchange_local(solvers):
    """The exchange of slab.exchange between contexts of one process, through host memory:
    every rank's side s goes to the neighbour's side 1 - s."""
    bufs = {}
    for r, s_ in enumerate(solvers):
        for side in (0, 1):
            if (s_.plan.shared_lo, s_.plan.shared_hi)[side]:
                b = s_.send[side]
                s_._export(side, b)
                bufs[(r, side)] = b.clone()
    for (r, side), b in bufs.items():
        p = solvers[r].plan
        peer = p.rank_lo if side == 0 else p.rank_hi
        solvers[peer]._import(1 - side, b)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("dim,periodic_axis,world", [
    (2, False, 3), (2, True, 2), (3, False, 2), (3, True, 3),
])
def test_slabs_match_the_oracle(precision, dim, periodic_axis, world):
    import torch
    w = _case(dim, periodic_axis, 7 + dim + world, with_src=not periodic_axis)
    ax = dim - 1
    plans = [slab.partition(w.n[ax], world, r, periodic_axis) for r in range(world)]
    solvers = [slab.SlabSolver(w, p, precision=precision, backend="gloo") for p in plans]
    nsteps = 6
    for _ in range(nsteps):
        for s_ in solvers:
            G.gks_step(s_.ctx, 1)
        _exchange_local(solvers)
    torch.cuda.synchronize()
    got = np.zeros((w.fields0.shape[0], int(np.prod(w.n))))
    for s_ in solvers:
        got[:, s_.ids[s_.owned]] = s_.read_owned()
    mesh = go.cartesian_mesh(w.n, w.lo, w.hi, w.bc)
    ref, _ = go.run(mesh, w.fields0, w.eps, None, w.cfl, nsteps, c=1.0, jz_mask=w.jz_mask,
                    src=w.src if w.jz_mask is not None else None)
    assert rel_l2(got, ref) <= TOL[precision], rel_l2(got, ref)
    # owned energies, summed in rank order, against the whole grid's
    e = 0.0
    for s_ in solvers:
        e += G.gks_energy(s_.ctx)
    e_ref = go.energy(mesh, go.fields_to_state(ref, dim), go.material_diag(w.eps, None))
    assert abs(e - e_ref) <= (1e-12 if precision == "fp64" else 1e-5) * e_ref
    for s_ in solvers:
        s_.close()


def test_transposed_exchange_is_the_adjoint_of_the_copy():
    """<P x, y> = <x, P^T y> with the library's halo calls on caller-owned state buffers (FP64):
    P copies owned layers into the neighbours' ghost layers, P^T adds ghost layers into the
    neighbours' owned layers."""
    import torch
    w = _case(3, True, 3, with_src=False)
    plans = [slab.partition(w.n[2], 3, r, True) for r in range(3)]
    solvers = [slab.SlabSolver(w, p, precision="fp64", backend="gloo") for p in plans]
    rng = np.random.default_rng(11)
    xs, ys, px, pty = [], [], [], []
    for s_ in solvers:
        nel, _ = G.gks_state_layout(s_.ctx)
        xs.append(torch.tensor(rng.standard_normal(nel), device="cuda"))
        ys.append(torch.tensor(rng.standard_normal(nel), device="cuda"))
        px.append(xs[-1].clone())
        pty.append(ys[-1].clone())
    dev = [[torch.empty(s_.send[0].numel(), dtype=torch.uint8, device="cuda") for _ in range(2)]
           for s_ in solvers]

    def run(src_layers, dst_layers, add, bufs):
        msgs = {}
        for r, s_ in enumerate(solvers):
            for side in (0, 1):
                G.gks_halo_export(s_.ctx, side, src_layers, bufs[r].data_ptr(), dev[r][side].data_ptr())
                msgs[(r, side)] = dev[r][side].cpu()
        for (r, side), b in msgs.items():
            p = solvers[r].plan
            peer = p.rank_lo if side == 0 else p.rank_hi
            d = b.cuda()
            G.gks_halo_import(solvers[peer].ctx, 1 - side, dst_layers, bufs[peer].data_ptr(),
                              d.data_ptr(), add)
        torch.cuda.synchronize()

    run(G.GKS_HALO_OWNED, G.GKS_HALO_GHOST, False, px)
    run(G.GKS_HALO_GHOST, G.GKS_HALO_OWNED, True, pty)
    lhs = sum(float(torch.dot(px[r], ys[r])) for r in range(3))
    # <x, P^T y> over owned layers: the owned range of each local state
    rhs = 0.0
    for r, s_ in enumerate(solvers):
        nel, _ = G.gks_state_layout(s_.ctx)
        ncomp = w.fields0.shape[0]
        per_comp = nel // ncomp
        nloc = s_.plan.n_local
        L = per_comp // nloc
        o0, o1 = s_.plan.own0 * L, (s_.plan.own0 + s_.plan.end - s_.plan.begin) * L
        x = xs[r].view(ncomp, per_comp)[:, o0:o1]
        y = pty[r].view(ncomp, per_comp)[:, o0:o1]
        rhs += float((x * y).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    for s_ in solvers:
        s_.close()
