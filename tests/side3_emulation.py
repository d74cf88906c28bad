"""CPU emulation (FP64 numpy) of the side-split 3-D step: the arithmetic the CUDA kernel does,
written with the generator's term lists, so that the tests can compare it with the oracle.

Test infrastructure: only the tests import this module."""
from __future__ import annotations

import numpy as np


def side_vectors(nt, A, v, d, ev, ed):
    """pl, pr, ql, qr [6][...] of cells with state v [6][...], raw differences d [3][6][...],
    ev [3][...], ed [3][3][...] for faces along axis A (nt: numeric term lists)."""
    def inp(name):
        if name.startswith("ev"):
            return ev[int(name[2:])]
        if name.startswith("ed"):
            j, m = name[2:].split("_")
            return ed[int(j)][int(m)]
        if name.startswith("v"):
            return v[int(name[1:])]
        j, m = name[1:].split("_")
        return d[int(j)][int(m)]

    zero = np.zeros_like(v[0])
    out = {}
    for part in ("EvP", "OdP", "EvQ", "OdQ"):
        out[part] = [sum((k * inp(x) for k, x in nt[A][(part, m)]), zero) for m in range(6)]
    pl = [out["EvP"][m] + out["OdP"][m] for m in range(6)]
    pr = [out["EvP"][m] - out["OdP"][m] for m in range(6)]
    ql = [out["EvQ"][m] + out["OdQ"][m] for m in range(6)]
    qr = [out["EvQ"][m] - out["OdQ"][m] for m in range(6)]
    return pl, pr, ql, qr


def _neighbour(n, periodic):
    """Index of the cell below and above every cell on an axis (wrap, or clamp = the
    non-reflecting ghost copy for the gradient)."""
    i = np.arange(n)
    if periodic:
        return (i - 1) % n, (i + 1) % n
    return np.maximum(i - 1, 0), np.minimum(i + 1, n - 1)


def step(nt, V, eps, periodic, jz_dt=None):
    """One side-split step.  V [6][nz][ny][nx] (x fastest), eps [nz][ny][nx], periodic[3] per
    axis (x, y, z), jz_dt [nz][ny][nx] = dt * J_z or None.  Returns V^{n+1}."""
    V = np.asarray(V, dtype=np.float64)
    n = V.shape[1:][::-1]                 # (nx, ny, nz)
    axis_np = (3, 2, 1)                   # numpy axis of x, y, z in V
    d = []
    for j in range(3):
        lo, hi = _neighbour(n[j], periodic[j])
        d.append(np.take(V, hi, axis=axis_np[j]) - np.take(V, lo, axis=axis_np[j]))
    ev = [eps * V[m] for m in range(3)]
    ed = [[eps * d[j][m] for m in range(3)] for j in range(3)]
    net = np.zeros_like(V)
    for A in range(3):
        pl, pr, ql, qr = side_vectors(nt, A, V, d, ev, ed)
        pl, pr, ql, qr = (np.stack(x) for x in (pl, pr, ql, qr))
        ax = axis_np[A]
        na = n[A]
        # face i+1/2 for i = 0..na-2 (interior), then the ends
        def sl(a, b):
            idx = [slice(None)] * 4
            idx[ax] = slice(a, b)
            return tuple(idx)

        def sl3(a, b):
            idx = [slice(None)] * 3
            idx[ax - 1] = slice(a, b)
            return tuple(idx)

        ie = 2.0 / (eps[sl3(0, na - 1)] + eps[sl3(1, na)])
        Fin = pl[sl(0, na - 1)] + pr[sl(1, na)] + ie * (ql[sl(0, na - 1)] + qr[sl(1, na)])
        if periodic[A]:
            ie_w = 2.0 / (eps[sl3(na - 1, na)] + eps[sl3(0, 1)])
            Fw = pl[sl(na - 1, na)] + pr[sl(0, 1)] + ie_w * (ql[sl(na - 1, na)] + qr[sl(0, 1)])
            Flo, Fhi = Fw, Fw
        else:
            Flo = pr[sl(0, 1)] + qr[sl(0, 1)] / eps[sl3(0, 1)]
            Fhi = pl[sl(na - 1, na)] + ql[sl(na - 1, na)] / eps[sl3(na - 1, na)]
        F = np.concatenate([Flo, Fin, Fhi], axis=ax)       # faces -1/2 .. na-1/2
        net += F[sl(1, na + 1)] - F[sl(0, na)]
    Vn = V - net
    for m in range(3):
        Vn[m] = V[m] - net[m] / eps
    if jz_dt is not None:
        Vn[2] = Vn[2] - jz_dt / eps
    return Vn
