"""GPU parity of the fused 3-D Cartesian step against the FP64 oracle (through the C ABI).

Tolerances (relative L2 over all components and cells): FP64 <= 1e-12, FP32 <= 2e-5."""
import numpy as np
import pytest

from oracle import gks_oracle as go
from paper_2412_16845_gb300 import workloads as wl
from paper_2412_16845_gb300.gks import GKSSolver
from tests.oracle_runs import oracle_block_step, rel_l2

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2412_16845_gb300 import build
    build.build()


def _random3(n, bc, seed, with_mu=False, with_src=False, h=None):
    rng = np.random.default_rng(seed)
    h = h or (1.0 / n[0],) * 3
    hi = tuple(h[d] * n[d] for d in range(3))
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
    return wl.CartWorkload(name="rand3", dim=3, n=n, lo=(0.0,) * 3, hi=hi, bc=bc, cfl=0.4,
                           steps=0, eps=eps, mu=mu, fields0=f, jz_mask=mask,
                           src=(1.0, 20.0, 0.02, 0.02), c_lattice=0.0)


def _gpu(w, steps, precision, kappa=0.0):
    s = GKSSolver.from_workload(w, precision=precision, kappa=kappa)
    s.step(steps)
    out = s.read_fields()
    info = s.info()
    s.close()
    return out, info


def _oracle(w, steps, kappa, c):
    mesh = go.cartesian_mesh(w.n, w.lo, w.hi, w.bc)
    return go.run(mesh, w.fields0, w.eps, w.mu, w.cfl, steps, kappa=kappa, c=c,
                  jz_mask=w.jz_mask, src=w.src if w.jz_mask is not None else None)[0]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("kappa", [0.0, 0.05, 1.0])
@pytest.mark.parametrize("case", [
    ((12, 10, 9), ("periodic",) * 6, False, False, None),
    ((33, 9, 7), ("nrbc",) * 6, True, True, None),
    ((7, 14, 11), ("nrbc", "nrbc", "periodic", "periodic", "nrbc", "nrbc"), False, True,
     (0.05, 0.03, 0.04)),
])
def test_random_grids(precision, kappa, case):
    """Small ragged grids, mixed boundaries, random eps and mu, scattered source, box cells,
    kappa in {0, 0.05, 1}; 8 steps.  (FP32 without mu runs the side-split kernel, whose CTA owns
    64 columns x 10 rows; the others run the staged-plane kernel.)"""
    n, bc, with_mu, with_src, h = case
    w = _random3(n, bc, seed=sum(n), with_mu=with_mu, with_src=with_src, h=h)
    out, info = _gpu(w, 8, precision, kappa)
    ref = _oracle(w, 8, kappa, info["c"])
    assert rel_l2(out, ref) <= TOL[precision], rel_l2(out, ref)


_WIDE_REF = {}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("kappa", [0.0, 0.05])
@pytest.mark.parametrize("case", [
    ((66, 31, 37), ("nrbc",) * 6, False),
    ((70, 23, 29), ("nrbc", "nrbc", "periodic", "periodic", "periodic", "periodic"), True),
])
def test_wide_ragged_grids(precision, kappa, case):
    """Grids spanning several CTAs in every direction: two x-tiles with a ragged second one,
    y > 28 rows (three to four row tiles, the last ragged), z split into several chunks; random
    eps, a scattered source on the first grid; 4 steps against the oracle."""
    n, bc, with_src = case
    w = _random3(n, bc, seed=sum(n) + 11, with_src=with_src)
    out, info = _gpu(w, 4, precision, kappa)
    key = (n, kappa)
    if key not in _WIDE_REF:
        _WIDE_REF[key] = _oracle(w, 4, kappa, info["c"])
    ref = _WIDE_REF[key]
    assert rel_l2(out, ref) <= TOL[precision], rel_l2(out, ref)


@pytest.mark.parametrize("n", [(1, 1, 1), (2, 3, 4), (5, 1, 3)])
@pytest.mark.parametrize("bc", ["periodic", "nrbc"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_degenerate_grids(n, bc, precision):
    w = _random3(n, (bc,) * 6, seed=3 + sum(n))
    out, info = _gpu(w, 5, precision)
    ref = _oracle(w, 5, 0.0, info["c"])
    assert rel_l2(out, ref) <= TOL[precision]


def test_sphere_workload_reduced():
    """The 256^3 sphere workload's structure at 20^3 (sphere, smoothed eps noise, incident
    pulse, non-reflecting boundary), 30 steps, FP64 and FP32 against the oracle."""
    w = wl.config3_sphere_3d(n=20, steps=30)
    ref = _oracle(w, 30, 0.0, 1.0)
    for prec in ("fp64", "fp32"):
        out, _ = _gpu(w, 30, prec)
        assert rel_l2(out, ref) <= TOL[prec], (prec, rel_l2(out, ref))


def test_full_size_sphere_sampled_fp32():
    """The 256^3 FP32 workload in the benchmark's launch configuration: after 20 steps, one more
    step is checked at 150 sampled cells (plus faces, corners and one whole z-column) against
    the oracle applied to the GPU's own state."""
    n = 256
    w = wl.config3_sphere_3d(n=n, steps=21)
    s = GKSSolver.from_workload(w, precision="fp32")
    s.step(20)
    before = s.read_fields()
    info = s.info()
    s.step(1)
    after = s.read_fields()
    s.close()
    rng = np.random.default_rng(5)
    cells = list(rng.choice(n ** 3, size=150, replace=False))
    cells += [0, n - 1, n * n - 1, n ** 3 - 1, n * n * (n // 2) + n * (n // 2) + 30]
    # a whole z-column at a corner of the side-split kernel's 64-column, 10-row tiles: it crosses
    # every boundary between the z-chunks the launch splits the grid into
    cells += [n * n * z + n * 10 + 64 for z in range(n)]
    ref = oracle_block_step(w, before, cells, info["dt"], 0.0, info["t"])
    scale = np.abs(before).max()
    assert np.abs(after[:, cells] - ref).max() <= 2e-6 * scale
