"""Discrete divergence and conservation on the periodic 2-D workload (64^2 unit square, oblique
plane wave k = 2 pi (2, 1) plus a Gaussian pulse, CFL 0.5, 200 steps), GPU FP64 through the C
ABI against the FP64 oracle.

- div_h H = (Hx(i+1) - Hx(i-1)) / (2h) + (Hy(j+1) - Hy(j-1)) / (2h), the central-difference
  divergence on the periodic grid, of the GPU fields equals the oracle's to 1e-12 relative to
  the size of its two terms (the update of Sec. 3.1 does not keep div_h H at zero: it is
  reported, not pinned to zero, and the bench prints its norm).
- sum_i |Omega_i| U_i (U = (eps Ez, Hx, Hy)) is conserved: on a periodic grid every face flux
  leaves one cell and enters another, so the total changes only by round-off."""
import numpy as np
import pytest

from oracle import gks_oracle as go
from paper_2412_16845_gb300 import workloads as wl
from paper_2412_16845_gb300.gks import GKSSolver
from tests.oracle_runs import oracle_cart_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2412_16845_gb300 import build
    build.build()


def div_h(fields, n, h):
    """Central-difference divergence of (Hx, Hy) on a periodic n x n grid, and the L2 norms of
    its two terms."""
    hx = fields[1].reshape(n, n)
    hy = fields[2].reshape(n, n)
    dx = (np.roll(hx, -1, axis=1) - np.roll(hx, 1, axis=1)) / (2 * h)
    dy = (np.roll(hy, -1, axis=0) - np.roll(hy, 1, axis=0)) / (2 * h)
    return dx + dy, np.linalg.norm(dx), np.linalg.norm(dy)


def test_divergence_matches_the_oracle_and_totals_are_conserved():
    n, steps = 64, 200
    w = wl.config1_periodic_tm(n)
    ref, _ = oracle_cart_run(w, steps)
    s = GKSSolver.from_workload(w, precision="fp64")
    u0 = s.read_fields()
    totals = []
    for k in range(4):
        s.step(steps // 4)
        f = s.read_fields()
        totals.append(f.sum(axis=1) * (1.0 / n) ** 2)    # eps = 1: U = V
    out = s.read_fields()
    s.close()
    h = 1.0 / n
    d_gpu, ax, ay = div_h(out, n, h)
    d_ref, _, _ = div_h(ref, n, h)
    scale = ax + ay
    assert np.linalg.norm(d_gpu - d_ref) <= 1e-12 * scale, (np.linalg.norm(d_gpu - d_ref), scale)
    # the divergence is a truncation-level quantity, far below its terms, but not round-off
    assert np.linalg.norm(d_gpu) <= 0.01 * scale      # 1.5e-3 in the oracle
    tot0 = u0.sum(axis=1) * h * h
    mag = (np.abs(u0).sum(axis=1) * h * h).max()
    for t in totals:
        assert np.abs(t - tot0).max() <= 1e-14 * max(1.0, mag) * 10, (t - tot0)
