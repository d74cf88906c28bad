"""GPU parity of the step with divergence cleaning (the PHM system of Sec. 2.1) against the
FP64 oracle, through the C ABI: 2-D TM (state Ez, Hx, Hy, psi) at CFL 0.4 and 3-D (state E, H,
phi, psi) at CFL 0.3, the cleaning system's stable ranges at lattice speed 1.

Tolerances (relative L2): FP64 <= 1e-12, FP32 <= 2e-5."""
import numpy as np
import pytest

from paper_2412_16845_gb300 import workloads as wl
from paper_2412_16845_gb300.gks import GKSSolver, GksError
from tests.oracle_runs import oracle_cart_run, rel_l2

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2412_16845_gb300 import build
    build.build()


def _w(nx, ny, bc, gamma, seed, with_src=False, chi=0.0):
    rng = np.random.default_rng(seed)
    hi = (1.0, ny / nx)
    x, y = wl.cell_centres_2d(nx, ny, hi=hi)
    f = np.stack([np.sin(2 * np.pi * x + 0.3) * np.cos(2 * np.pi * y),
                  0.5 * np.cos(2 * np.pi * (x + y)), np.sin(2 * np.pi * y - 0.2),
                  0.3 * np.sin(2 * np.pi * (x - y))])
    f += 0.1 * rng.standard_normal(f.shape)
    eps = rng.uniform(1.0, 4.0, nx * ny)
    mask = None
    if with_src:
        mask = np.zeros(nx * ny)
        k = max(1, nx * ny // 20)
        mask[rng.choice(nx * ny, size=k, replace=False)] = rng.uniform(-3, 3, k)
    return wl.CartWorkload(name="phm2", dim=2, n=(nx, ny), lo=(0.0, 0.0), hi=hi, bc=bc,
                           cfl=0.4, steps=0, eps=eps, mu=None, fields0=f, jz_mask=mask,
                           src=(1.0, 20.0, 0.02, 0.02), c_lattice=0.0, phm=(chi, gamma))


def _gpu(w, steps, precision, kappa):
    s = GKSSolver.from_workload(w, precision=precision, kappa=kappa)
    s.step(steps)
    out, info = s.read_fields(), s.info()
    s.close()
    return out, info


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("kappa", [0.0, 0.05])
@pytest.mark.parametrize("case", [
    (45, 37, ("nrbc",) * 4, 0.7, True),
    (131, 70, ("periodic",) * 4, 1.0, False),        # several strips and row chunks
    (70, 33, ("pec", "nrbc", "periodic", "periodic"), 0.5, True),
    (33, 70, ("nrbc", "pec", "pec", "nrbc"), 1.5, False),   # gamma > 1: lattice speed gamma
    (2, 3, ("pec",) * 4, 0.8, False),
])
def test_phm_2d(precision, kappa, case):
    nx, ny, bc, gamma, with_src = case
    w = _w(nx, ny, bc, gamma, seed=nx * 3 + ny, with_src=with_src, chi=0.4)
    steps = 20
    out, info = _gpu(w, steps, precision, kappa)
    assert out.shape[0] == 4
    ref, rinfo = oracle_cart_run(w, steps, kappa=kappa, c=info["c"])
    assert info["c"] == max(1.0 / np.sqrt(w.eps.min()), gamma)
    assert rel_l2(out, ref) <= TOL[precision], rel_l2(out, ref)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", [
    (127, 130, ("nrbc", "nrbc", "periodic", "periodic"), 1.0, True),   # strips, chunks, wrap
    (64, 47, ("nrbc",) * 4, 0.7, True),       # two strips, the second one column wide
    (33, 9, ("nrbc",) * 4, 1.3, False),       # high-x face on the second half of lane 1's pair
    (63, 2, ("nrbc",) * 4, 0.5, True),        # one strip, two rows
    (1, 5, ("nrbc",) * 4, 0.8, False),        # one column
    (200, 3, ("nrbc", "nrbc", "periodic", "periodic"), 1.0, False),   # periodic y on 3 rows
])
def test_phm_2d_staged_shapes(precision, case):
    """Shapes spanning the staged FP32 cleaning kernel's strips (63 columns, a lane's two cells
    32 apart) and row chunks, against the oracle (FP64 runs the scalar kernel on the same
    cases); kappa = 0.05, 12 steps."""
    nx, ny, bc, gamma, with_src = case
    w = _w(nx, ny, bc, gamma, seed=nx + 5 * ny, with_src=with_src, chi=0.4)
    out, info = _gpu(w, 12, precision, 0.05)
    ref, _ = oracle_cart_run(w, 12, kappa=0.05, c=info["c"])
    assert rel_l2(out, ref) <= TOL[precision], rel_l2(out, ref)


def test_phm_cleaning_wave_against_exact():
    """The standing cleaning wave of Sec. 2.1 (H_x = sin(2 pi x) initially, psi = 0, gamma =
    0.5) on the GPU: H_x = sin(2 pi x) cos(2 pi gamma t), psi = -cos(2 pi x) sin(2 pi gamma t)
    within the scheme's error at 128 cells, Ez and Hy staying zero."""
    n = 128
    x, y = wl.cell_centres_2d(n, 4, hi=(1.0, 4.0 / n))
    f = np.zeros((4, n * 4))
    f[1] = np.sin(2 * np.pi * x)
    w = wl.CartWorkload(name="cw", dim=2, n=(n, 4), lo=(0.0, 0.0), hi=(1.0, 4.0 / n),
                        bc=("periodic",) * 4, cfl=0.4, steps=0, eps=np.ones(n * 4), mu=None,
                        fields0=f, c_lattice=1.0, phm=(0.0, 0.5))
    s = GKSSolver.from_workload(w, precision="fp64")
    dt = s.info()["dt"]
    steps = int(round(0.4 / dt))
    s.step(steps)
    out = s.read_fields()
    s.close()
    t = steps * dt
    ex = np.sin(2 * np.pi * x) * np.cos(2 * np.pi * 0.5 * t)
    ep = -np.cos(2 * np.pi * x) * np.sin(2 * np.pi * 0.5 * t)
    assert np.sqrt(np.mean((out[1] - ex) ** 2 + (out[3] - ep) ** 2)) <= 3e-4
    assert np.max(np.abs(out[[0, 2]])) <= 1e-13


def test_phm_rejects_mu_and_adjoint():
    import torch
    from paper_2412_16845_gb300.gks import gks_adjoint_step, gks_set_objective, gks_state_layout
    w = _w(8, 8, ("nrbc",) * 4, 0.5, seed=1)
    s = GKSSolver.from_workload(w, precision="fp64")
    with pytest.raises(GksError):
        s.set_materials(np.ones(64), np.full(64, 2.0))
    gks_set_objective(s.ctx, None, None)
    n, _ = gks_state_layout(s.ctx)
    a = torch.zeros(n, dtype=torch.float64, device="cuda")
    b = torch.zeros_like(a)
    with pytest.raises(GksError):
        gks_adjoint_step(s.ctx, None, None, a.data_ptr(), b.data_ptr(), None, False)
    s.close()
    w3 = _w3(4, 4, 4, ("nrbc",) * 6, (0.5, 0.5), seed=2)
    s = GKSSolver.from_workload(w3, precision="fp32")
    with pytest.raises(GksError):
        s.set_materials(np.ones(64), np.full(64, 2.0))
    s.close()


# ------------------------------------------------------------------------------------------
# 3-D: state (Ex, Ey, Ez, Hx, Hy, Hz, phi, psi), CFL 0.3


def _w3(nx, ny, nz, bc, phm, seed, with_src=False):
    rng = np.random.default_rng(seed)
    h = 1.0 / nx
    hi = (1.0, ny * h, nz * h)
    idx = np.arange(nx * ny * nz)
    x = (idx % nx + 0.5) * h
    y = ((idx // nx) % ny + 0.5) * h
    z = (idx // (nx * ny) + 0.5) * h
    f = np.stack([np.sin(2 * np.pi * (x + k * y) + 0.4 * k) * np.cos(2 * np.pi * (z - 0.1 * k))
                  for k in range(8)])
    f += 0.1 * rng.standard_normal(f.shape)
    eps = rng.uniform(1.0, 4.0, nx * ny * nz)
    mask = None
    if with_src:
        mask = np.zeros(nx * ny * nz)
        k = max(1, mask.size // 20)
        mask[rng.choice(mask.size, size=k, replace=False)] = rng.uniform(-3, 3, k)
    return wl.CartWorkload(name="phm3", dim=3, n=(nx, ny, nz), lo=(0.0,) * 3, hi=hi, bc=bc,
                           cfl=0.3, steps=0, eps=eps, mu=None, fields0=f, jz_mask=mask,
                           src=(1.0, 20.0, 0.02, 0.02), c_lattice=0.0, phm=phm)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("kappa", [0.0, 0.05])
@pytest.mark.parametrize("case", [
    (13, 11, 9, ("nrbc",) * 6, (0.7, 0.4), True),
    (34, 15, 7, ("periodic",) * 6, (1.0, 1.0), False),    # two tiles along x and along y
    (9, 8, 10, ("pec", "nrbc", "periodic", "periodic", "nrbc", "pec"), (0.5, 0.8), True),
    (6, 7, 5, ("nrbc", "pec", "pec", "nrbc", "pec", "pec"), (1.5, 0.3), False),   # chi > 1
    (2, 3, 2, ("pec",) * 6, (0.6, 0.9), False),
])
def test_phm_3d(precision, kappa, case):
    nx, ny, nz, bc, phm, with_src = case
    w = _w3(nx, ny, nz, bc, phm, seed=nx * 7 + ny + nz, with_src=with_src)
    steps = 12
    out, info = _gpu(w, steps, precision, kappa)
    assert out.shape == (8, nx * ny * nz)
    assert info["c"] == max(1.0 / np.sqrt(w.eps.min()), *phm)
    ref, _ = oracle_cart_run(w, steps, kappa=kappa, c=info["c"])
    assert rel_l2(out, ref) <= TOL[precision], rel_l2(out, ref)


_WIDE_PHM_REF = {}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("kappa", [0.0, 0.05])
@pytest.mark.parametrize("case", [
    (65, 23, 19, ("nrbc",) * 6, (1.0, 1.0), True),
    (61, 31, 17, ("nrbc", "nrbc", "periodic", "periodic", "periodic", "periodic"), (0.7, 0.4),
     False),
])
def test_phm_3d_wide_ragged_grids(precision, kappa, case):
    """The cleaning kernel on grids spanning several CTAs in every direction: three x-tiles of
    its 30-column interior with a ragged last one, y over 20 rows (three or four 10-row tiles,
    the last ragged), z split into several chunks; a scattered source on the first grid; 4 steps
    against the oracle."""
    nx, ny, nz, bc, phm, with_src = case
    w = _w3(nx, ny, nz, bc, phm, seed=nx + 3 * ny + nz, with_src=with_src)
    out, info = _gpu(w, 4, precision, kappa)
    key = (nx, ny, nz, kappa)
    if key not in _WIDE_PHM_REF:
        _WIDE_PHM_REF[key] = oracle_cart_run(w, 4, kappa=kappa, c=info["c"])[0]
    assert rel_l2(out, _WIDE_PHM_REF[key]) <= TOL[precision], rel_l2(out, _WIDE_PHM_REF[key])


def test_phm_3d_energy_includes_potentials():
    """gks_energy with cleaning: 1/2 sum |Omega| (eps |E|^2 + |H|^2 + phi^2 + psi^2)."""
    w = _w3(10, 9, 8, ("nrbc",) * 6, (0.5, 0.5), seed=4)
    s = GKSSolver.from_workload(w, precision="fp64")
    e = s.energy()
    s.close()
    f = w.fields0
    vol = (1.0 / 10) ** 3
    ref = 0.5 * vol * np.sum(w.eps * (f[0:3] ** 2).sum(0) + (f[3:8] ** 2).sum(0))
    assert abs(e - ref) <= 1e-12 * ref


def test_phm_3d_cleaning_waves_against_exact():
    """Two standing cleaning waves of Sec. 2.1 at once on a periodic 64 x 64 x 2 grid: E_x =
    sin(2 pi x) with chi = 0.7 (exact E_x = sin(2 pi x) cos(2 pi chi t), phi = -cos(2 pi x)
    sin(2 pi chi t)) and H_y = sin(2 pi y) with gamma = 0.5 (psi likewise along y).  Both
    fields are curl free, so the Maxwell part stays at rest: every other component stays 0."""
    n = 64
    h = 1.0 / n
    idx = np.arange(n * n * 2)
    x = (idx % n + 0.5) * h
    y = ((idx // n) % n + 0.5) * h
    f = np.zeros((8, idx.size))
    f[0] = np.sin(2 * np.pi * x)
    f[4] = np.sin(2 * np.pi * y)
    chi, gam = 0.7, 0.5
    w = wl.CartWorkload(name="cw3", dim=3, n=(n, n, 2), lo=(0.0,) * 3, hi=(1.0, 1.0, 2 * h),
                        bc=("periodic",) * 6, cfl=0.3, steps=0, eps=np.ones(idx.size), mu=None,
                        fields0=f, c_lattice=1.0, phm=(chi, gam))
    s = GKSSolver.from_workload(w, precision="fp64")
    dt = s.info()["dt"]
    steps = int(round(0.4 / dt))
    s.step(steps)
    out = s.read_fields()
    s.close()
    t = steps * dt
    err = np.sqrt(np.mean((out[0] - np.sin(2 * np.pi * x) * np.cos(2 * np.pi * chi * t)) ** 2 +
                          (out[6] + np.cos(2 * np.pi * x) * np.sin(2 * np.pi * chi * t)) ** 2 +
                          (out[4] - np.sin(2 * np.pi * y) * np.cos(2 * np.pi * gam * t)) ** 2 +
                          (out[7] + np.cos(2 * np.pi * y) * np.sin(2 * np.pi * gam * t)) ** 2))
    assert err <= 3e-3, err
    assert np.max(np.abs(out[[1, 2, 3, 5]])) <= 1e-13
