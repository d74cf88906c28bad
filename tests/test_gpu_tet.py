"""GPU parity of the tetrahedral GKS step against the FP64 oracle (through the C ABI).

Tolerances (relative L2, volume-weighted): FP64 <= 1e-12, FP32 <= 2e-5."""
import numpy as np
import pytest

from oracle import gks_oracle as go
from paper_2412_16845_gb300 import workloads as wl
from paper_2412_16845_gb300.gks import GKSSolver

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2412_16845_gb300 import build
    build.build()


def vrel(a, b, vol):
    num = np.sqrt(np.sum(vol * (a - b) ** 2))
    return float(num / np.sqrt(np.sum(vol * b ** 2)))


def _rand_tets(m, seed, jitter=0.1, with_mu=False, with_src=False):
    rng = np.random.default_rng(seed)
    vert, tet = wl.kuhn_tet_mesh(m, jitter, rng)
    cen = vert[tet].mean(axis=1)
    f = np.stack([np.sin(2 * np.pi * (cen[:, 0] + 0.1 * c)) * np.cos(2 * np.pi * cen[:, 1] + c)
                  for c in range(6)])
    f += 0.1 * rng.standard_normal(f.shape)
    nt = tet.shape[0]
    eps = rng.uniform(1.0, 4.0, nt)
    mu = rng.uniform(1.0, 2.0, nt) if with_mu else None
    mask = None
    if with_src:
        mask = np.zeros(nt)
        k = max(1, nt // 20)
        mask[rng.choice(nt, size=k, replace=False)] = rng.uniform(-3, 3, k)
    return vert, tet, eps, mu, f, mask


def _gpu(vert, tet, eps, mu, f, mask, steps, prec, kappa, src=(1.0, 20.0, 0.02, 0.02)):
    s = GKSSolver.from_tets(vert, tet, 0.4, precision=prec, kappa=kappa)
    s.set_materials(eps, mu)
    s.write_fields(f)
    if mask is not None:
        s.set_source(mask, *src)
    s.step(steps)
    out = s.read_fields()
    info = s.info()
    s.close()
    return out, info


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("kappa", [0.0, 0.05])
@pytest.mark.parametrize("case", [(3, False, False), (4, True, True), (5, False, True)])
def test_random_tet_meshes(precision, kappa, case):
    """Jittered Kuhn meshes, random eps (and mu), scattered source, 10 steps.  The meshes hold
    162, 384 and 750 tets: one, two and three 256-thread blocks per pass, the last one partly
    full."""
    m, with_mu, with_src = case
    vert, tet, eps, mu, f, mask = _rand_tets(m, 40 + m, with_mu=with_mu, with_src=with_src)
    out, info = _gpu(vert, tet, eps, mu, f, mask, 10, precision, kappa)
    mesh = go.tet_mesh(vert, tet)
    dt = go.time_step(mesh, 0.4, 1.0)
    assert abs(info["dt"] - dt) <= 1e-14 * dt
    ref, _ = go.run(mesh, f, eps, mu, 0.4, 10, kappa=kappa, c=1.0, jz_mask=mask,
                    src=(1.0, 20.0, 0.02, 0.02) if mask is not None else None)
    assert vrel(out, ref, mesh.vol) <= TOL[precision], vrel(out, ref, mesh.vol)


def test_sphere_tet_workload_reduced():
    """The 1.57M-tet workload's structure with 8^3 hexes (3072 tets): jittered, eps = 4 sphere,
    incident pulse, non-reflecting boundary, 25 steps, FP64 and FP32."""
    w = wl.config4_tets(m=8, steps=25)
    mesh = go.tet_mesh(w.vert, w.tet)
    ref, _ = go.run(mesh, w.fields0, w.eps, None, w.cfl, 25, c=1.0)
    for prec in ("fp64", "fp32"):
        s = GKSSolver.from_tet_workload(w, precision=prec)
        s.step(25)
        out = s.read_fields()
        s.close()
        assert vrel(out, ref, mesh.vol) <= TOL[prec], (prec, vrel(out, ref, mesh.vol))


def test_energy_on_tets():
    vert, tet, eps, mu, f, mask = _rand_tets(3, 7, with_mu=True)
    s = GKSSolver.from_tets(vert, tet, 0.4, precision="fp64")
    s.set_materials(eps, mu)
    s.write_fields(f)
    s.step(2)
    e = s.energy()
    out = s.read_fields()
    s.close()
    mesh = go.tet_mesh(vert, tet)
    ref = go.energy(mesh, go.fields_to_state(out, 3), go.material_diag(eps, mu))
    assert abs(e - ref) <= 1e-13 * ref


def _neighbours(tet):
    """Face neighbours of every tet (user ids), from shared sorted vertex triples."""
    nt = tet.shape[0]
    opp = [(1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2)]
    tri = np.concatenate([np.sort(tet[:, list(o)], axis=1) for o in opp])
    owner = np.tile(np.arange(nt), 4)
    order = np.lexsort((tri[:, 2], tri[:, 1], tri[:, 0]))
    ts, os_ = tri[order], owner[order]
    same = np.all(ts[1:] == ts[:-1], axis=1)
    a, b = os_[:-1][same], os_[1:][same]
    nb = [[] for _ in range(nt)]
    for x, y in zip(a.tolist(), b.tolist()):
        nb[x].append(y)
        nb[y].append(x)
    return nb


def test_full_size_tets_sampled_fp32():
    """The 64^3 x 6 = 1,572,864-tet FP32 workload: after 10 steps, one more step is checked at
    60 sampled tets against the oracle run on the sub-mesh of tets within two face-hops of each
    sample (the stencil of the step), using the GPU's own state."""
    w = wl.config4_tets(m=64, steps=11)
    s = GKSSolver.from_tet_workload(w, precision="fp32")
    s.step(10)
    before = s.read_fields()
    info = s.info()
    s.step(1)
    after = s.read_fields()
    s.close()
    nb = _neighbours(w.tet)
    rng = np.random.default_rng(11)
    samples = list(rng.choice(w.tet.shape[0], size=60, replace=False)) + [0, w.tet.shape[0] - 1]
    C = go.time_coefficients(info["dt"], 0.0)
    worst = 0.0
    scale = np.abs(before).max()
    for c in samples:
        ring = {int(c)}
        frontier = {int(c)}
        for _ in range(2):
            frontier = {y for x in frontier for y in nb[x]} - ring
            ring |= frontier
        sub = np.array(sorted(ring))                    # user order kept: same face orientation
        mesh = go.tet_mesh(w.vert, w.tet[sub])
        V = go.fields_to_state(before[:, sub], 3)
        m = go.material_diag(w.eps[sub], None)
        Vn = go.step(mesh, V, m, info["dt"], C, 1.0)
        k = int(np.searchsorted(sub, c))
        worst = max(worst, float(np.abs(go.state_to_fields(Vn[k:k + 1], 3)[:, 0] - after[:, c]).max()))
    assert worst <= 2e-6 * scale, worst / scale
