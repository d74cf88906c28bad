"""gks_energy_noalloc: the energy of caller-owned device arrays without any allocation.

It serves callers that cannot allocate device memory (a framework holding the device memory in
its own pool, a hot loop that cannot pay for an allocation, code without a gks context).  The
check: through the C ABI, two calls in a row give the energy that gks_energy computes for the
same fields, within the tolerance of the energy test (1e-13 relative).  This file runs last."""
import ctypes

import numpy as np
import pytest

from paper_2412_16845_gb300 import workloads as wl
from paper_2412_16845_gb300.gks import (GKS_E_ARG, GKS_FP32, GKS_FP64, GKSSolver, GksError,
                                        gks_energy_noalloc, load_library)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2412_16845_gb300 import build
    build.build()


def _cases():
    rng = np.random.default_rng(12)
    n2 = (37, 29)
    f2 = rng.standard_normal((3, n2[0] * n2[1]))
    w2 = wl.CartWorkload(name="e2", dim=2, n=n2, lo=(0.0, 0.0), hi=(1.0, 29 / 37), bc=("nrbc",) * 4,
                         cfl=0.5, steps=0, eps=rng.uniform(1, 3, f2.shape[1]),
                         mu=rng.uniform(1, 2, f2.shape[1]), fields0=f2)
    n3 = (11, 9, 7)
    f3 = rng.standard_normal((6, int(np.prod(n3))))
    w3 = wl.CartWorkload(name="e3", dim=3, n=n3, lo=(0.0,) * 3, hi=(1.0, 9 / 11, 7 / 11),
                         bc=("nrbc",) * 6, cfl=0.4, steps=0, eps=rng.uniform(1, 3, f3.shape[1]),
                         mu=None, fields0=f3)
    # many 4096-cell blocks with a partly filled last one: 300 x 301 = 90,300 cells (23 blocks)
    # and 64^3 = 262,144 cells (64 full blocks)
    nb = (300, 301)
    fb = rng.standard_normal((3, nb[0] * nb[1]))
    wb = wl.CartWorkload(name="e2b", dim=2, n=nb, lo=(0.0, 0.0), hi=(1.0, 301 / 300),
                         bc=("nrbc",) * 4, cfl=0.5, steps=0, eps=rng.uniform(1, 3, fb.shape[1]),
                         mu=None, fields0=fb)
    nc = (64, 64, 64)
    fc = rng.standard_normal((6, int(np.prod(nc))))
    wc = wl.CartWorkload(name="e3b", dim=3, n=nc, lo=(0.0,) * 3, hi=(1.0,) * 3, bc=("nrbc",) * 6,
                         cfl=0.4, steps=0, eps=rng.uniform(1, 3, fc.shape[1]),
                         mu=rng.uniform(1, 2, fc.shape[1]), fields0=fc)
    return [w2, w3, wb, wc]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_noalloc_energy_matches_gks_energy(precision, k):
    import torch
    w = _cases()[k]
    s = GKSSolver.from_workload(w, precision=precision)
    s.step(2)
    ref = s.energy()
    fields = s.read_fields()          # the state the context holds, in user order
    s.close()
    dt = torch.float64 if precision == "fp64" else torch.float32
    dev = torch.device("cuda", 0)
    f_d = torch.as_tensor(fields, dtype=dt).to(dev).contiguous()
    e_d = torch.as_tensor(w.eps, dtype=dt).to(dev)
    m_d = None if w.mu is None else torch.as_tensor(w.mu, dtype=dt).to(dev)
    out = torch.full((1,), -1.0, dtype=torch.float64, device=dev)
    vol = float(np.prod([(w.hi[a] - w.lo[a]) / w.n[a] for a in range(w.dim)]))
    stream = torch.cuda.current_stream().cuda_stream
    prec = GKS_FP64 if precision == "fp64" else GKS_FP32
    got = []
    for _ in range(2):                 # two calls in a row share the fixed scratch
        gks_energy_noalloc(prec, w.dim, fields.shape[1], vol, f_d.data_ptr(), e_d.data_ptr(),
                           0 if m_d is None else m_d.data_ptr(), out.data_ptr(), stream)
        torch.cuda.synchronize()
        got.append(float(out.item()))
        out.fill_(-1.0)
    for g in got:
        assert abs(g - ref) <= 1e-13 * abs(ref), (g, ref)


def test_noalloc_rejects_oversized_and_bad_arguments():
    import torch
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(GksError) as ei:
        gks_energy_noalloc(GKS_FP64, 2, 33554432 + 1, 1.0, x.data_ptr(), x.data_ptr(), 0,
                           out.data_ptr())
    assert ei.value.status == GKS_E_ARG
    with pytest.raises(GksError):
        gks_energy_noalloc(GKS_FP64, 4, 2, 1.0, x.data_ptr(), x.data_ptr(), 0, out.data_ptr())
    with pytest.raises(GksError):
        gks_energy_noalloc(GKS_FP64, 2, 2, 1.0, 0, x.data_ptr(), 0, out.data_ptr())
