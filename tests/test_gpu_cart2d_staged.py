"""GPU parity of the staged 2-D TM step (FP32, mu = 1; non-reflecting, PEC or periodic-y sides:
rows staged in shared memory by tensor copies, a lane's two cells 32 columns apart, 63 columns per
warp) against the FP64 oracle, relative L2 <= 2e-5.

Shapes span the strip and chunk structure of that kernel: widths below, at and past one
63-column strip and ragged against it, high-x boundary faces on either half of a lane's pair,
heights of one or two rows and heights that split a strip into several row chunks with an odd
last chunk; PEC walls on either axis (mirror rows and columns in the staged rows); sources,
periodic y (with the two-row wrap), rectangular cells."""
import numpy as np
import pytest

from oracle import gks_oracle as go
from paper_2412_16845_gb300 import workloads as wl
from paper_2412_16845_gb300.gks import GKSSolver
from tests.oracle_runs import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2412_16845_gb300 import build
    build.build()


def _workload(nx, ny, ybc, seed, with_src, hy_ratio=1.0, xbc="nrbc"):
    rng = np.random.default_rng(seed)
    hi = (1.0, hy_ratio * ny / nx)
    x, y = wl.cell_centres_2d(nx, ny, hi=hi)
    f = np.stack([np.sin(2 * np.pi * x + 0.3) * np.cos(2 * np.pi * y),
                  0.5 * np.cos(2 * np.pi * (x + y)), np.sin(2 * np.pi * y - 0.2)])
    f += 0.1 * rng.standard_normal(f.shape)
    eps = rng.uniform(1.0, 4.0, nx * ny)
    mask = None
    if with_src:
        k = max(1, nx * ny // 25)
        mask = np.zeros(nx * ny)
        mask[rng.choice(nx * ny, size=k, replace=False)] = rng.uniform(-3, 3, k)
    return wl.CartWorkload(name="staged", dim=2, n=(nx, ny), lo=(0.0, 0.0), hi=hi,
                           bc=(xbc, xbc, ybc, ybc), cfl=0.5, steps=0, eps=eps, mu=None,
                           fields0=f, jz_mask=mask, src=(1.0, 20.0, 0.02, 0.02), c_lattice=0.0)


@pytest.mark.parametrize("nx,ny,ybc,src,hy", [
    (64, 47, "nrbc", True, 1.0),      # two strips, the second one column wide; 6 row chunks
    (59, 9, "nrbc", False, 0.7),      # one strip, its last cells past the grid
    (63, 2, "nrbc", True, 1.0),       # exactly one strip, two rows
    (127, 130, "nrbc", True, 1.3),    # three strips, many chunks, odd last chunk
    (33, 40, "nrbc", True, 1.0),      # high-x face on the second half of lane 1's pair
    (32, 5, "nrbc", False, 1.0),      # high-x face on the second half of lane 0's pair
    (1, 7, "nrbc", False, 1.0),       # one column: both x faces on the same cell
    (3, 1, "nrbc", True, 1.0),        # one row: both y faces on the same cell
    (200, 3, "periodic", True, 1.0),  # periodic y on three rows (wrap of two rows)
    (7, 300, "periodic", False, 0.5), # periodic y, tall and narrow
    (45, 2, "periodic", False, 1.0),  # periodic y on two rows
])
def test_staged_step_matches_the_oracle(nx, ny, ybc, src, hy):
    w = _workload(nx, ny, ybc, seed=nx + 1000 * ny, with_src=src, hy_ratio=hy)
    steps = 17
    s = GKSSolver.from_workload(w, precision="fp32")
    s.step(steps)
    out = s.read_fields()
    c = s.info()["c"]
    s.close()
    mesh = go.cartesian_mesh(w.n, w.lo, w.hi, w.bc)
    ref, _ = go.run(mesh, w.fields0, w.eps, None, w.cfl, steps, c=c, jz_mask=w.jz_mask,
                    src=w.src if w.jz_mask is not None else None)
    assert rel_l2(out, ref) <= 2e-5, rel_l2(out, ref)


@pytest.mark.parametrize("nx,ny,xbc,ybc,src", [
    (64, 47, "pec", "pec", True),          # closed box: mirror rows and columns, corners
    (33, 9, "pec", "nrbc", False),         # PEC x walls, high wall on lane 1's second cell
    (63, 2, "nrbc", "pec", True),          # PEC y walls on two rows
    (2, 7, "pec", "pec", False),           # two columns: the mirrors span the whole grid
    (127, 130, "pec", "periodic", True),   # three strips, chunks, periodic y
    (32, 5, "pec", "nrbc", False),         # high wall on lane 0's second cell
])
def test_staged_step_pec_walls(nx, ny, xbc, ybc, src):
    """PEC walls (Sec. 5.5) through the staged kernel: rows and columns past a wall are mirror
    images written into the staged rows, the wall faces interior faces against them."""
    w = _workload(nx, ny, ybc, seed=nx + 77 * ny, with_src=src, xbc=xbc)
    steps = 17
    s = GKSSolver.from_workload(w, precision="fp32")
    s.step(steps)
    out = s.read_fields()
    c = s.info()["c"]
    s.close()
    mesh = go.cartesian_mesh(w.n, w.lo, w.hi, w.bc)
    ref, _ = go.run(mesh, w.fields0, w.eps, None, w.cfl, steps, c=c, jz_mask=w.jz_mask,
                    src=w.src if w.jz_mask is not None else None)
    assert rel_l2(out, ref) <= 2e-5, rel_l2(out, ref)


def test_staged_window_steps_match_the_oracle_inside():
    """Windowed steps through the staged kernel (rows and strips of a window that starts and
    ends inside the grid): after k steps the cells at least 2k cells inside the window equal
    the whole-grid oracle run."""
    from paper_2412_16845_gb300.gks import gks_step_window
    nx, ny = 190, 110
    w = _workload(nx, ny, "nrbc", seed=5, with_src=True)
    s = GKSSolver.from_workload(w, precision="fp32")
    k = 3
    gks_step_window(s.ctx, k, 61, 170, 21, 96)
    out = s.read_fields()
    c = s.info()["c"]
    s.close()
    mesh = go.cartesian_mesh(w.n, w.lo, w.hi, w.bc)
    ref, _ = go.run(mesh, w.fields0, w.eps, None, w.cfl, k, c=c, jz_mask=w.jz_mask, src=w.src)
    o = out.reshape(3, ny, nx)[:, 21 + 2 * k:96 - 2 * k, 61 + 2 * k:170 - 2 * k]
    r = ref.reshape(3, ny, nx)[:, 21 + 2 * k:96 - 2 * k, 61 + 2 * k:170 - 2 * k]
    assert rel_l2(o, r) <= 2e-5, rel_l2(o, r)
