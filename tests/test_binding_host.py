"""Host-side marshalling of the Python binding (no GPU): the descriptor GKSSolver builds from a
SolverSpec, captured by replacing the create call."""
import pytest

from paper_2412_16845_gb300 import gks


@pytest.fixture
def captured(monkeypatch):
    seen = {}

    def fake_create(desc):
        seen["desc"] = desc
        return None                  # no context: close() and __del__ then do nothing

    monkeypatch.setattr(gks, "gks_create_mesh", fake_create)
    return seen


def _spec(**kw):
    base = dict(dim=3, n=(8, 6, 4), lo=(0.0, 0.0, 0.0), hi=(1.0, 0.75, 0.5),
                bc=("nrbc", "pec", "periodic", "periodic", "pec", "nrbc"), cfl=0.3)
    base.update(kw)
    return gks.SolverSpec(**base)


def test_descriptor_carries_grid_boundaries_and_options(captured):
    s = gks.GKSSolver(_spec(precision="fp64", kappa=0.05, c_lattice=1.5, phm=(0.7, 0.4),
                            limiter="vanleer"))
    d = captured["desc"]
    assert (d.dim, d.kind, d.precision) == (3, gks.GKS_CARTESIAN, gks.GKS_FP64)
    assert list(d.n) == [8, 6, 4] and list(d.hi) == [1.0, 0.75, 0.5]
    assert list(d.bc) == [gks.GKS_BC_NONREFLECTING, gks.GKS_BC_PEC, gks.GKS_BC_PERIODIC,
                          gks.GKS_BC_PERIODIC, gks.GKS_BC_PEC, gks.GKS_BC_NONREFLECTING]
    assert (d.cfl, d.tau_over_dt, d.c_lattice) == (0.3, 0.05, 1.5)
    assert (d.chi, d.gamma, d.limiter) == (0.7, 0.4, gks.GKS_LIMITER_VAN_LEER)
    assert s.ncomp == 8 and s.ncell == 8 * 6 * 4


@pytest.mark.parametrize("dim,phm,ncomp", [(2, None, 3), (2, (0.0, 1.0), 4), (3, None, 6),
                                           (3, (1.0, 0.0), 8), (2, (0.0, 0.0), 3)])
def test_component_count(captured, dim, phm, ncomp):
    spec = _spec(dim=dim, n=(8, 6, 4)[:dim], lo=(0.0,) * dim, hi=(1.0,) * dim,
                 bc=("nrbc",) * (2 * dim), phm=phm)
    s = gks.GKSSolver(spec)
    d = captured["desc"]
    assert s.ncomp == ncomp
    assert d.limiter == gks.GKS_LIMITER_NONE
    assert (d.chi, d.gamma) == ((phm or (0.0, 0.0))[0], (phm or (0.0, 0.0))[1])


def test_cleaning_fields_without_potentials_are_padded(captured, monkeypatch):
    import numpy as np
    seen = {}
    monkeypatch.setattr(gks, "gks_write_fields",
                        lambda ctx, f, t0: seen.__setitem__("f", np.array(f).ravel()))
    s = gks.GKSSolver(_spec(phm=(0.5, 0.5)))          # 3-D: 8 components
    n = s.ncell
    f6 = np.arange(6 * n, dtype=float).reshape(6, n)
    s.write_fields(f6)
    assert seen["f"].shape == (8 * n,)
    assert np.array_equal(seen["f"][:6 * n], f6.ravel()) and not seen["f"][6 * n:].any()
    f8 = np.ones((8, n))
    s.write_fields(f8)
    assert np.array_equal(seen["f"], f8.ravel())
    with pytest.raises(ValueError):
        s.write_fields(np.ones((5, n)))
