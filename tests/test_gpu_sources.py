"""GPU parity of the oscillating-dipole workloads of Sec. 5.4 (continuous-wave current source,
gks_set_source_cw) against the FP64 oracle, through the C ABI.

Tolerances (relative L2): FP64 <= 1e-12, FP32 <= 2e-5."""
import pytest

from paper_2412_16845_gb300 import workloads as wl
from paper_2412_16845_gb300.gks import GKSSolver
from tests.oracle_runs import oracle_cart_run, rel_l2

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2412_16845_gb300 import build
    build.build()


def _run_gpu(w, steps, precision, kappa):
    s = GKSSolver.from_workload(w, precision=precision, kappa=kappa)
    s.step(steps)
    out, info = s.read_fields(), s.info()
    s.close()
    return out, info


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("two", [False, True])
def test_dipole_workloads(precision, two):
    """The oscillating-dipole workloads of Sec. 5.4 (continuous-wave source, gks_set_source_cw):
    one dipole on 100 x 100 and two on 100 x 50, to t = 0.5, against the oracle."""
    w = wl.dipole_tm(n=100 if not two else 50, two=two, t_end=0.5)
    out, info = _run_gpu(w, w.steps, precision, 0.0)
    ref, rinfo = oracle_cart_run(w, w.steps, c=info["c"])
    assert info["dt"] == rinfo["dt"]
    assert rel_l2(out, ref) <= TOL[precision], rel_l2(out, ref)
