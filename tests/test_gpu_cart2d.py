"""GPU parity of the fused 2-D TM step against the FP64 oracle (through the C ABI).

Tolerances (relative L2 over all components and cells): FP64 <= 1e-12, FP32 <= 2e-5."""
import math

import numpy as np
import pytest

from oracle import gks_oracle as go
from paper_2412_16845_gb300 import workloads as wl
from paper_2412_16845_gb300.gks import GKSSolver, GksError, SolverSpec, GKS_E_NONFINITE, GKS_E_ARG
from tests.oracle_runs import oracle_block_step, oracle_cart_run, rel_l2

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2412_16845_gb300 import build
    build.build()


def _random_workload(nx, ny, bc, seed, with_mu=False, with_src=False, hx=None):
    rng = np.random.default_rng(seed)
    hi = (1.0, (ny / nx) if hx is None else hx * ny)
    x, y = wl.cell_centres_2d(nx, ny, hi=hi)
    f = np.stack([np.sin(2 * np.pi * x + 0.3) * np.cos(2 * np.pi * y),
                  0.5 * np.cos(2 * np.pi * (x + y)), np.sin(2 * np.pi * y - 0.2)])
    f += 0.1 * rng.standard_normal(f.shape)
    eps = rng.uniform(1.0, 4.0, nx * ny)
    mu = rng.uniform(1.0, 2.0, nx * ny) if with_mu else None
    mask = None
    if with_src:
        mask = np.zeros(nx * ny)
        mask[rng.choice(nx * ny, size=max(1, nx * ny // 20), replace=False)] = \
            rng.uniform(-3, 3, max(1, nx * ny // 20))
    return wl.CartWorkload(name="rand", dim=2, n=(nx, ny), lo=(0.0, 0.0), hi=hi, bc=bc,
                           cfl=0.5, steps=0, eps=eps, mu=mu, fields0=f, jz_mask=mask,
                           src=(1.0, 20.0, 0.02, 0.02), c_lattice=0.0)


def _gpu_run(w, steps, precision, kappa=0.0, dt=None):
    s = GKSSolver.from_workload(w, precision=precision, kappa=kappa)
    if dt is not None:
        s.set_dt(dt)
    s.step(steps)
    out = s.read_fields()
    info = s.info()
    s.close()
    return out, info


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_periodic_plane_wave_and_pulse_64(precision):
    """64x64 periodic vacuum, oblique wave + seeded pulse, CFL 0.5, 200 steps."""
    w = wl.config1_periodic_tm(64)
    ref, rinfo = oracle_cart_run(w, 200)
    out, info = _gpu_run(w, 200, precision)
    assert info["dt"] == rinfo["dt"]
    assert rel_l2(out, ref) <= TOL[precision], rel_l2(out, ref)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("kappa", [0.0, 0.05, 1.0, 1e3])
@pytest.mark.parametrize("case", [
    (45, 37, ("nrbc",) * 4, True, True, None),
    (70, 33, ("periodic",) * 2 + ("nrbc",) * 2, False, True, None),
    (33, 70, ("nrbc",) * 2 + ("periodic",) * 2, True, False, 0.013),
])
def test_ragged_grids_materials_source(precision, kappa, case):
    """Ragged tiles (sizes not multiples of the 32x16 tile), mixed boundaries, random eps and
    mu, a scattered source, rectangular cells, every kappa; 25 steps."""
    nx, ny, bc, with_mu, with_src, hx = case
    w = _random_workload(nx, ny, bc, seed=nx * 100 + ny, with_mu=with_mu, with_src=with_src,
                         hx=hx)
    steps = 25
    out, info = _gpu_run(w, steps, precision, kappa=kappa)
    # lattice speed chosen by the library: max_i 1/sqrt(eps_i mu_i) (sub-characteristic)
    c = float(np.max(1.0 / np.sqrt(w.eps * (1.0 if w.mu is None else w.mu))))
    assert abs(info["c"] - c) <= 1e-15 * c
    mesh = go.cartesian_mesh(w.n, w.lo, w.hi, w.bc)
    dt = go.time_step(mesh, w.cfl, c)
    assert abs(info["dt"] - dt) <= 1e-15 * dt
    ref, _ = go.run(mesh, w.fields0, w.eps, w.mu, w.cfl, steps, kappa=kappa, c=c,
                    jz_mask=w.jz_mask, src=w.src if w.jz_mask is not None else None)
    assert rel_l2(out, ref) <= TOL[precision], rel_l2(out, ref)


@pytest.mark.parametrize("n", [(1, 1), (2, 3), (3, 1), (1, 5), (33, 17)])
@pytest.mark.parametrize("bc", ["periodic", "nrbc"])
def test_degenerate_grids(n, bc):
    """Grids of one or a few cells in a direction (the stencil wraps onto itself, or every face
    is a boundary face)."""
    w = _random_workload(n[0], n[1], (bc,) * 4, seed=7 + n[0] + 10 * n[1])
    out, info = _gpu_run(w, 6, "fp64")
    ref, _ = oracle_cart_run(w, 6, c=info["c"])
    assert rel_l2(out, ref) <= 1e-12


def test_cylinders_source_reduced_fp32_and_fp64():
    """The 4096^2 cylinder workload's structure at 128^2 (cylinders, line source, non-reflecting
    boundary), 200 steps (t = 0.78, the whole source pulse), FP32 and FP64 against the
    oracle."""
    w = wl.config2_cylinders_tm(n=128, steps=200)
    ref, rinfo = oracle_cart_run(w, 200)
    for prec in ("fp64", "fp32"):
        out, info = _gpu_run(w, 200, prec)
        assert abs(info["t"] - rinfo["t"]) < 1e-12
        assert rel_l2(out, ref) <= TOL[prec], (prec, rel_l2(out, ref))
    assert np.abs(ref).max() > 1e-3   # the source did inject a field


def test_energy_matches_oracle():
    w = _random_workload(50, 40, ("nrbc",) * 4, seed=3, with_mu=True)
    w.eps[0] = 1.0
    w.mu[0] = 1.0
    s = GKSSolver.from_workload(w, precision="fp64")
    s.step(3)
    e = s.energy()
    out = s.read_fields()
    s.close()
    mesh = go.cartesian_mesh(w.n, w.lo, w.hi, w.bc)
    ref = go.energy(mesh, go.fields_to_state(out, 2), go.material_diag(w.eps, w.mu))
    assert abs(e - ref) <= 1e-13 * ref


def test_full_size_cylinders_sampled_fp32():
    """The 4096^2 FP32 workload in the launch configuration the benchmark times: after 60 steps
    one more step is checked at 300 sampled cells (plus every source cell of one row band)
    against the oracle applied to the GPU's own state."""
    w = wl.config2_cylinders_tm(n=4096, steps=61)
    s = GKSSolver.from_workload(w, precision="fp32")
    s.step(60)
    before = s.read_fields()
    t = s.info()["t"]
    dt = s.info()["dt"]
    s.step(1)
    after = s.read_fields()
    s.close()
    rng = np.random.default_rng(99)
    n = 4096
    cells = list(rng.choice(n * n, size=300, replace=False))
    i_src = w.extra["i_src"]
    cells += [i_src + n * j for j in (0, 1, 2047, 4094, 4095)]
    cells += [0, n - 1, n * (n - 1), n * n - 1]                  # corners
    cells += [i_src + 1 + n * 2048, i_src - 1 + n * 2048]
    # cells near cylinders
    for cx, cy, r, _ in w.extra["cylinders"][:4]:
        cells.append(int(cx * n) + n * int(cy * n))
        cells.append(int((cx + r) * n) + n * int(cy * n))
    ref = oracle_block_step(w, before, cells, dt, 0.0, t)
    got = after[:, cells]
    scale = np.abs(before).max()
    assert scale > 0
    assert np.abs(got - ref).max() <= 2e-6 * scale + 1e-30, np.abs(got - ref).max() / scale


def test_nonfinite_input_is_reported():
    w = _random_workload(20, 20, ("nrbc",) * 4, seed=1)
    s = GKSSolver.from_workload(w, precision="fp32")
    f = w.fields0.copy()
    f[0, 17] = np.nan
    s.write_fields(f)
    s.step(2)
    with pytest.raises(GksError) as ei:
        s.read_fields()
    assert ei.value.status == GKS_E_NONFINITE
    s.write_fields(w.fields0)   # a fresh write clears the flag
    s.step(1)
    s.read_fields()
    s.close()


def test_bad_materials_rejected_before_any_work():
    w = _random_workload(8, 8, ("nrbc",) * 4, seed=2)
    s = GKSSolver.from_workload(w, precision="fp32")
    eps = w.eps.copy()
    eps[3] = 0.0
    with pytest.raises(GksError) as ei:
        s.set_materials(eps)
    assert ei.value.status == GKS_E_ARG
    s.close()
