"""The folded interior-face flux of the divergence-cleaning system (csrc/gks_phm3.cuh, written
by paper_2412_16845_gb300/codegen.py) against the FP64 oracle, on the CPU.

* The committed header is exactly what the generator writes.
* With the generator's numeric coefficients, the folded flux (every term a coefficient a + b ie
  times a side sum, difference or eps-weighted sum/difference, ie = 2/(eps_l + eps_r)) equals
  the oracle's literal D3Q4 face flux of Sec. 3.1 for the cleaning system of Sec. 2.1 (in the
  face frame, times dt/h) on random interior faces: random values and derivatives of all eight
  components on both sides, unequal permittivities, several kappa, chi and gamma (including
  gamma = 0) and lattice speeds."""
import numpy as np
import pytest

from oracle import gks_oracle as go

sp = pytest.importorskip("sympy")
from paper_2412_16845_gb300 import codegen  # noqa: E402


@pytest.fixture(scope="module")
def terms():
    return codegen.derive_phm()


def test_header_is_generated(terms):
    with open(codegen.PHM_HEADER) as f:
        committed = f.read()
    assert committed == codegen.emit_phm(terms), \
        "regenerate: python -m paper_2412_16845_gb300.codegen"


@pytest.mark.parametrize("kappa", [0.0, 0.05, 1.0])
@pytest.mark.parametrize("chi,gam,c", [(1.0, 1.0, 1.0), (1.3, 0.7, 1.7), (2.0, 0.0, 1.2)])
def test_folded_flux_equals_the_oracle(terms, kappa, chi, gam, c):
    rng = np.random.default_rng(int(100 * kappa + 10 * chi + gam))
    h, dt = 0.07, 0.02
    C = go.time_coefficients(dt, kappa * dt)
    flux = codegen.phm_numeric(terms, C, h, c, chi, gam)
    for _ in range(5):
        sides = []
        for _s in range(2):
            sides.append({"v": rng.standard_normal(8), "dn": rng.standard_normal(8),
                          "dt": rng.standard_normal(8), "dw": rng.standard_normal(8),
                          "eps": rng.uniform(1.0, 5.0)})
        l, r = sides
        got = np.array(flux(l, r))
        G = [np.stack([s["dn"], s["dt"], s["dw"]])[None] for s in sides]
        ml = go.material_diag(np.array([l["eps"]]), None, 8)
        mr = go.material_diag(np.array([r["eps"]]), None, 8)
        ref = go.face_flux_local(l["v"][None], G[0], ml, r["v"][None], G[1], mr,
                                 np.array([False]), C, dt, c, 3, phm=(chi, gam))[0] * dt / h
        assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max()), (got, ref)
