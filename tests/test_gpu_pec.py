"""GPU parity of the PEC wall boundary (Sec. 5.5 wall conditions, mirror ghost) against the FP64
oracle, through the C ABI: 2-D TM and 3-D Cartesian grids (PEC on every side and mixed with
non-reflecting and periodic sides) and tetrahedral PEC cavities.

Tolerances (relative L2): FP64 <= 1e-12, FP32 <= 2e-5."""
import numpy as np
import pytest

from oracle import gks_oracle as go
from paper_2412_16845_gb300 import workloads as wl
from paper_2412_16845_gb300.gks import GKSSolver, GksError
from tests.oracle_runs import oracle_cart_run, rel_l2

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2412_16845_gb300 import build
    build.build()


def _w2(nx, ny, bc, seed, with_mu=False, with_src=False):
    rng = np.random.default_rng(seed)
    hi = (1.0, ny / nx)
    x, y = wl.cell_centres_2d(nx, ny, hi=hi)
    f = np.stack([np.sin(2 * np.pi * x + 0.3) * np.cos(2 * np.pi * y),
                  0.5 * np.cos(2 * np.pi * (x + y)), np.sin(2 * np.pi * y - 0.2)])
    f += 0.1 * rng.standard_normal(f.shape)
    eps = rng.uniform(1.0, 4.0, nx * ny)
    mu = rng.uniform(1.0, 2.0, nx * ny) if with_mu else None
    mask = None
    if with_src:
        mask = np.zeros(nx * ny)
        k = max(1, nx * ny // 20)
        mask[rng.choice(nx * ny, size=k, replace=False)] = rng.uniform(-3, 3, k)
    return wl.CartWorkload(name="pec2", dim=2, n=(nx, ny), lo=(0.0, 0.0), hi=hi, bc=bc,
                           cfl=0.5, steps=0, eps=eps, mu=mu, fields0=f, jz_mask=mask,
                           src=(1.0, 20.0, 0.02, 0.02), c_lattice=0.0)


def _run_gpu(w, steps, precision, kappa):
    s = GKSSolver.from_workload(w, precision=precision, kappa=kappa)
    s.step(steps)
    out, info = s.read_fields(), s.info()
    s.close()
    return out, info


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("kappa", [0.0, 0.05])
@pytest.mark.parametrize("case", [
    (45, 37, ("pec",) * 4, True, True),
    (131, 70, ("pec",) * 4, False, False),               # several strips and row chunks
    (70, 33, ("pec", "nrbc", "periodic", "periodic"), False, True),
    (33, 70, ("nrbc", "pec", "pec", "nrbc"), True, False),
    (2, 3, ("pec",) * 4, False, False),                  # the smallest PEC axes
])
def test_pec_2d(precision, kappa, case):
    nx, ny, bc, with_mu, with_src = case
    w = _w2(nx, ny, bc, seed=nx * 7 + ny, with_mu=with_mu, with_src=with_src)
    steps = 20
    out, info = _run_gpu(w, steps, precision, kappa)
    ref, rinfo = oracle_cart_run(w, steps, kappa=kappa, c=info["c"])
    assert rel_l2(out, ref) <= TOL[precision], rel_l2(out, ref)


def test_pec_2d_cavity_mode_matches_periodic():
    """The paper's TM cavity mode (Sec. 5.2) on the GPU: the PEC box and the periodic box give
    the same fields (FP64, to rounding), as they do in the oracle."""
    N = 64
    x, y = wl.cell_centres_2d(N, N)
    f = np.zeros((3, N * N))
    f[0] = np.sin(8 * np.pi * x) * np.sin(8 * np.pi * y)
    outs = []
    for bc in (("pec",) * 4, ("periodic",) * 4):
        w = wl.CartWorkload(name="cav", dim=2, n=(N, N), lo=(0.0, 0.0), hi=(1.0, 1.0), bc=bc,
                            cfl=0.5, steps=0, eps=np.ones(N * N), mu=None, fields0=f)
        outs.append(_run_gpu(w, 100, "fp64", 0.0)[0])
    assert np.max(np.abs(outs[0] - outs[1])) <= 1e-12


def _w3(n, bc, seed, with_mu=False, with_src=False):
    rng = np.random.default_rng(seed)
    h = 1.0 / n[0]
    hi = tuple(h * n[d] for d in range(3))
    x, y, z = wl.cell_centres_3d(*n, hi=hi)
    f = np.stack([np.sin(2 * np.pi * (x + c * 0.1)) * np.cos(2 * np.pi * (y - z) + c)
                  for c in range(6)])
    f += 0.1 * rng.standard_normal(f.shape)
    ncell = int(np.prod(n))
    eps = rng.uniform(1.0, 3.0, ncell)
    mu = rng.uniform(1.0, 2.0, ncell) if with_mu else None
    mask = None
    if with_src:
        mask = np.zeros(ncell)
        k = max(1, ncell // 30)
        mask[rng.choice(ncell, size=k, replace=False)] = rng.uniform(-3, 3, k)
    return wl.CartWorkload(name="pec3", dim=3, n=n, lo=(0.0,) * 3, hi=hi, bc=bc, cfl=0.4,
                           steps=0, eps=eps, mu=mu, fields0=f, jz_mask=mask,
                           src=(1.0, 20.0, 0.02, 0.02), c_lattice=0.0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("kappa", [0.0, 0.05])
@pytest.mark.parametrize("case", [
    ((12, 10, 9), ("pec",) * 6, False, True),
    ((33, 17, 7), ("pec",) * 6, True, False),            # several CTAs in x and y
    ((9, 14, 11), ("pec", "nrbc", "periodic", "periodic", "nrbc", "pec"), False, True),
    ((2, 3, 2), ("pec",) * 6, False, False),
])
def test_pec_3d(precision, kappa, case):
    n, bc, with_mu, with_src = case
    w = _w3(n, bc, seed=sum(n) + 5, with_mu=with_mu, with_src=with_src)
    steps = 8
    out, info = _run_gpu(w, steps, precision, kappa)
    mesh = go.cartesian_mesh(w.n, w.lo, w.hi, w.bc)
    ref = go.run(mesh, w.fields0, w.eps, w.mu, w.cfl, steps, kappa=kappa, c=info["c"],
                 jz_mask=w.jz_mask, src=w.src if w.jz_mask is not None else None)[0]
    assert rel_l2(out, ref) <= TOL[precision], rel_l2(out, ref)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("kappa", [0.0, 0.05])
@pytest.mark.parametrize("with_mu", [False, True])
def test_pec_tets(precision, kappa, with_mu):
    """A jittered Kuhn-tet box with PEC walls on every boundary face, random eps (and mu)."""
    rng = np.random.default_rng(77)
    vert, tet = wl.kuhn_tet_mesh(4, 0.1, rng)
    cen = vert[tet].mean(axis=1)
    f = np.stack([np.sin(2 * np.pi * (cen[:, 0] + 0.1 * c)) * np.cos(2 * np.pi * cen[:, 1] + c)
                  for c in range(6)])
    f += 0.1 * rng.standard_normal(f.shape)
    nt = tet.shape[0]
    eps = rng.uniform(1.0, 4.0, nt)
    mu = rng.uniform(1.0, 2.0, nt) if with_mu else None
    s = GKSSolver.from_tets(vert, tet, 0.4, precision=precision, kappa=kappa, bc="pec")
    s.set_materials(eps, mu)
    s.write_fields(f)
    s.step(10)
    out = s.read_fields()
    s.close()
    mesh = go.tet_mesh(vert, tet, bc="pec")
    ref, _ = go.run(mesh, f, eps, mu, 0.4, 10, kappa=kappa, c=1.0)
    num = np.sqrt(np.sum(mesh.vol * (out - ref) ** 2))
    err = float(num / np.sqrt(np.sum(mesh.vol * ref ** 2)))
    assert err <= TOL[precision], err


def test_pec_adjoint_is_unsupported():
    from paper_2412_16845_gb300.gks import gks_adjoint_step, gks_set_objective, gks_state_layout
    import torch
    w = _w2(8, 8, ("pec",) * 4, seed=1)
    s = GKSSolver.from_workload(w, precision="fp64")
    gks_set_objective(s.ctx, None, None)
    n, _ = gks_state_layout(s.ctx)
    a = torch.zeros(n, dtype=torch.float64, device="cuda")
    b = torch.zeros_like(a)
    with pytest.raises(GksError):
        gks_adjoint_step(s.ctx, None, None, a.data_ptr(), b.data_ptr(), None, False)
    s.close()

