"""The hand-written adjoint of the 2-D TM step and the eps-gradient of the probe objective.

Checks: the transpose identity <L x, y> = <x, L^T y> (FP64, 1e-13); the gradient against the
oracle's complex-step derivative (exact to round-off) and against central finite differences of
the GPU's FP64 forward; FP32 against FP64; the torch.autograd wrapper."""
import numpy as np
import pytest

from oracle import gks_oracle as go
from paper_2412_16845_gb300 import workloads as wl
from paper_2412_16845_gb300.gks import (GKSSolver, gks_adjoint_step, gks_copy_state,
                                        gks_load_state, gks_state_layout, gks_set_objective)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2412_16845_gb300 import build
    build.build()


def _grid(nx, ny, bc, seed):
    rng = np.random.default_rng(seed)
    x, y = wl.cell_centres_2d(nx, ny, hi=(1.0, ny / nx))
    f = rng.standard_normal((3, nx * ny))
    eps = rng.uniform(1.0, 3.0, nx * ny)
    return wl.CartWorkload(name="adj", dim=2, n=(nx, ny), lo=(0.0, 0.0), hi=(1.0, ny / nx),
                           bc=bc, cfl=0.5, steps=0, eps=eps, mu=None, fields0=f)


@pytest.mark.parametrize("bc", [("nrbc",) * 4, ("periodic",) * 4,
                                ("periodic", "periodic", "nrbc", "nrbc")])
@pytest.mark.parametrize("kappa", [0.0, 0.05, 1.0])
@pytest.mark.parametrize("n", [(37, 23), (5, 3), (131, 70)])
def test_transpose_identity(bc, kappa, n):
    import torch
    w = _grid(n[0], n[1], bc, 3 + n[0])
    s = GKSSolver.from_workload(w, precision="fp64", kappa=kappa)
    gks_set_objective(s.ctx, None, None)
    elems, _ = gks_state_layout(s.ctx)
    # random x, y in the padded layout (padding entries stay zero)
    rng = np.random.default_rng(9)
    pad = torch.zeros(elems, dtype=torch.float64, device="cuda")
    gks_copy_state(s.ctx, pad.data_ptr())            # the layout of the written fields
    mask = torch.zeros(elems, dtype=torch.float64, device="cuda")
    s.write_fields(np.ones((3, w.ncell)))
    gks_copy_state(s.ctx, mask.data_ptr())
    x = torch.as_tensor(rng.standard_normal(elems), device="cuda") * mask
    y = torch.as_tensor(rng.standard_normal(elems), device="cuda") * mask
    gks_load_state(s.ctx, x.data_ptr(), 0)
    s.step(1)
    Lx = torch.empty_like(x)
    gks_copy_state(s.ctx, Lx.data_ptr())
    LTy = torch.zeros_like(y)
    gks_adjoint_step(s.ctx, None, None, y.data_ptr(), LTy.data_ptr(), None, False)
    torch.cuda.synchronize()
    a = float((Lx * y).sum())
    b = float((x * LTy * mask).sum())
    s.close()
    assert abs(a - b) <= 1e-13 * max(abs(a), float((x * x).sum()) ** 0.5 * float((y * y).sum()) ** 0.5), (a, b)


def _design_workload(nx=24, ny=20, steps=30, seed=5):
    rng = np.random.default_rng(seed)
    x, y = wl.cell_centres_2d(nx, ny, hi=(1.0, ny / nx))
    h = 1.0 / nx
    f = np.zeros((3, nx * ny))
    f[0] = np.exp(-((x - 0.3) ** 2 + (y - 0.4) ** 2) / (2 * 0.08 ** 2))
    eps = np.ones(nx * ny)
    ii, jj = np.arange(8, 16), np.arange(6, 14)
    design = (jj[:, None] * nx + ii[None, :]).ravel()
    eps[design] = rng.uniform(1.0, 3.0, design.size)
    probe = np.nonzero((x - 0.6) ** 2 + (y - 0.45) ** 2 <= 0.1 ** 2)[0]
    mask = np.zeros(nx * ny)
    mask[(np.arange(nx * ny) % nx) == 3] = 1.0 / h
    return wl.CartWorkload(name="design", dim=2, n=(nx, ny), lo=(0.0, 0.0), hi=(1.0, ny / nx),
                           bc=("nrbc",) * 4, cfl=0.5, steps=steps, eps=eps, mu=None, fields0=f,
                           jz_mask=mask, src=(1.0, 4.0, 0.1, 0.1), probe=probe,
                           design=design.astype(np.int64))


def _oracle_J(w, eps):
    mesh = go.cartesian_mesh(w.n, w.lo, w.hi, w.bc)
    _, info = go.run(mesh, w.fields0, eps, None, w.cfl, w.steps, c=1.0, jz_mask=w.jz_mask,
                     src=w.src, probe=w.probe)
    return info["J"]


def test_gradient_matches_oracle_complex_step():
    """FP64 adjoint gradient = the oracle's complex-step derivative (Im J(eps + i h e_d)/h)."""
    from paper_2412_16845_gb300.adjoint import DesignProblem
    w = _design_workload()
    prob = DesignProblem(w, precision="fp64", checkpoint_every=7)
    J, g = prob.value_and_grad(w.eps[w.design])
    prob.close()
    Jo = _oracle_J(w, w.eps)
    assert abs(J - Jo) <= 1e-12 * abs(Jo)
    picks = [0, 5, 17, 33, 50, 63]
    for k in picks:
        e = w.eps.astype(complex)
        e[w.design[k]] += 1e-30j
        ref = _oracle_J(w, e).imag / 1e-30
        assert abs(g[k] - ref) <= 1e-9 * max(abs(ref), 1e-12 * abs(J)), (k, g[k], ref)


def test_gradient_fd_fp64_and_fp32_agree():
    """Central differences of the GPU FP64 forward, and the FP32 adjoint within 1e-3."""
    from paper_2412_16845_gb300.adjoint import DesignProblem
    w = _design_workload(nx=40, ny=32, steps=60, seed=6)
    w.design = w.design  # same design box definition scaled to the grid
    p64 = DesignProblem(w, precision="fp64")
    J, g64 = p64.value_and_grad(w.eps[w.design])
    base = w.eps[w.design].copy()
    rng = np.random.default_rng(1)
    for k in rng.choice(w.design.size, size=6, replace=False):
        h = 1e-5
        ep = base.copy(); ep[k] += h
        em = base.copy(); em[k] -= h
        fd = (p64.forward(ep, keep_checkpoints=False) - p64.forward(em, keep_checkpoints=False)) / (2 * h)
        assert abs(fd - g64[k]) <= 1e-6 * np.abs(g64).max(), (k, fd, g64[k])
    p64.close()
    p32 = DesignProblem(w, precision="fp32")
    J32, g32 = p32.value_and_grad(base)
    p32.close()
    assert abs(J32 - J) <= 1e-4 * abs(J)
    assert np.linalg.norm(g32 - g64) <= 1e-3 * np.linalg.norm(g64)


def test_autograd_function():
    import torch
    from paper_2412_16845_gb300.adjoint import DesignProblem, GKSEnergyObjective
    w = _design_workload()
    prob = DesignProblem(w, precision="fp64", checkpoint_every=5)
    e = torch.tensor(w.eps[w.design], dtype=torch.float64, device="cuda", requires_grad=True)
    J = GKSEnergyObjective.apply(e, prob)
    J.backward()
    _, g = prob.value_and_grad(w.eps[w.design])
    prob.close()
    assert np.allclose(e.grad.cpu().numpy(), g, rtol=1e-12, atol=0)


def test_full_size_design_gradient_fd_16_cells():
    """The 2048^2 inverse-design workload (2000 steps, 512^2 design region, probe disc r = 0.02,
    checkpoints every 45 steps): the FP32 adjoint gradient against central differences (h = 1e-3)
    of the FP64 forward at 16 seeded design cells, relative L2 <= 1e-3 over the 16 cells."""
    from paper_2412_16845_gb300.adjoint import DesignProblem
    w = wl.config5_design_tm(n=2048, steps=2000)
    e0 = w.eps[w.design].copy()
    p32 = DesignProblem(w, precision="fp32", checkpoint_every=45)
    J32, g32 = p32.value_and_grad(e0)
    p32.close()
    p64 = DesignProblem(w, precision="fp64", checkpoint_every=45)
    rng = np.random.default_rng(20241216 + 5)
    # seeded cells inside the probe's region of influence (central part of the design box)
    i0, i1, j0, j1 = w.extra["design_box"]
    ks = []
    while len(ks) < 16:
        k = int(rng.integers(0, w.design.size))
        if k not in ks:
            ks.append(k)
    fd = []
    for k in ks:
        ep = e0.copy(); ep[k] += 1e-3
        em = e0.copy(); em[k] -= 1e-3
        fd.append((p64.forward(ep, keep_checkpoints=False) -
                   p64.forward(em, keep_checkpoints=False)) / 2e-3)
    p64.close()
    fd = np.array(fd)
    ad = g32[ks]
    assert J32 > 0 and np.abs(fd).max() > 0
    assert np.linalg.norm(ad - fd) <= 1e-3 * np.linalg.norm(fd), (ad, fd)


def test_materials_box_equals_full_update():
    """gks_set_materials_box on a sub-rectangle gives bit-identical steps to gks_set_materials
    with the same eps; its argument and state errors."""
    from paper_2412_16845_gb300.gks import GksError, gks_set_materials_box
    w = _design_workload(nx=40, ny=32, steps=20, seed=8)
    rng = np.random.default_rng(9)
    x0, x1, y0, y1 = 5, 29, 7, 19
    new = w.eps.copy().reshape(32, 40)
    new[y0:y1, x0:x1] = rng.uniform(1.0, 4.0, (y1 - y0, x1 - x0))
    out = []
    for use_box in (False, True):
        for prec in ("fp64", "fp32"):
            s = GKSSolver.from_workload(w, precision=prec, c_lattice=1.0)
            if use_box:
                gks_set_materials_box(s.ctx, x0, x1, y0, y1, new[y0:y1, x0:x1].copy())
            else:
                s.set_materials(new.ravel())
            s.write_fields(w.fields0)
            s.step(20)
            out.append(s.read_fields())
            s.close()
    assert np.array_equal(out[0], out[2]) and np.array_equal(out[1], out[3])
    s = GKSSolver.from_workload(w, precision="fp32", c_lattice=0.0)   # automatic lattice speed
    with pytest.raises(GksError):
        gks_set_materials_box(s.ctx, 0, 2, 0, 2, np.ones(4))
    s.close()
    s = GKSSolver.from_workload(w, precision="fp32", c_lattice=1.0)
    with pytest.raises(GksError):
        gks_set_materials_box(s.ctx, 30, 41, 0, 2, np.ones(22))
    with pytest.raises(GksError):
        gks_set_materials_box(s.ctx, 0, 2, 0, 2, np.array([1.0, 0.0, 1.0, 1.0]))
    s.close()


def test_design_below_lattice_speed_rejected():
    from paper_2412_16845_gb300.adjoint import DesignProblem
    w = _design_workload()
    prob = DesignProblem(w, precision="fp32")
    e = w.eps[w.design].copy()
    e[3] = 0.5
    with pytest.raises(ValueError):
        prob.forward(e)
    prob.close()


def test_reset_objective():
    """gks_reset_objective needs an objective (GKS_E_STATE before gks_set_objective) and sets the
    accumulated J back to zero; a run restarted from a stored state then repeats J exactly."""
    import torch
    from paper_2412_16845_gb300.gks import (GksError, gks_copy_state, gks_load_state,
                                            gks_objective, gks_reset_objective,
                                            gks_set_objective, gks_state_layout)
    w = _design_workload()
    s = GKSSolver.from_workload(w, precision="fp64")
    with pytest.raises(GksError):
        gks_reset_objective(s.ctx)
    gks_set_objective(s.ctx, w.probe, w.design)
    n, _ = gks_state_layout(s.ctx)
    v0 = torch.empty(n, dtype=torch.float64, device="cuda")
    gks_copy_state(s.ctx, v0.data_ptr())
    s.step(10)
    J1 = gks_objective(s.ctx)
    assert J1 > 0
    gks_reset_objective(s.ctx)
    assert gks_objective(s.ctx) == 0.0
    gks_load_state(s.ctx, v0.data_ptr(), 0)
    s.step(10)
    assert gks_objective(s.ctx) == J1
    s.close()
