"""GPU parity of the 2-D TM step with divergence cleaning (the PHM system of Sec. 2.1: state
Ez, Hx, Hy, psi; gamma > 0) against the FP64 oracle, through the C ABI.  CFL 0.4 (the cleaning
system's stable range at lattice speed 1).

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


def test_phm_rejects_mu_adjoint_and_3d():
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
    w3 = wl.CartWorkload(name="p3", dim=3, n=(4, 4, 4), lo=(0.0,) * 3, hi=(1.0,) * 3,
                         bc=("nrbc",) * 6, cfl=0.3, steps=0, eps=np.ones(64), mu=None,
                         fields0=np.zeros((6, 64)), phm=(0.5, 0.5))
    with pytest.raises(GksError):
        GKSSolver.from_workload(w3, precision="fp64")
