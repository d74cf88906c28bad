"""Helpers that run the FP64 oracle on the same seeded workloads the GPU path gets, and compare.

Test infrastructure: only the tests import this module."""
from __future__ import annotations

import numpy as np

from oracle import gks_oracle as go


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.sqrt(np.sum(b * b))
    return float(np.sqrt(np.sum((a - b) ** 2)) / (den if den > 0 else 1.0))


def oracle_cart_run(w, steps, kappa=0.0, dt=None, c=1.0):
    """Run the oracle on a Cartesian workload (w from paper_2412_16845_gb300.workloads)."""
    mesh = go.cartesian_mesh(w.n, w.lo, w.hi, w.bc)
    src = w.src if w.jz_mask is not None else None
    return go.run(mesh, w.fields0, w.eps, w.mu, w.cfl, steps, kappa=kappa, c=c,
                  jz_mask=w.jz_mask, src=src, dt=dt,
                  waveform=getattr(w, "waveform", "gauss_sine"), phm=getattr(w, "phm", None),
                  limiter=getattr(w, "limiter", None))


def oracle_block_step(w, fields, cells, dt, kappa, t, c=1.0):
    """One oracle step evaluated only at ``cells`` (user ids) of a non-periodic Cartesian
    workload, from the state ``fields`` [ncomp][ncell] at time t.

    Each sampled cell is updated on the block of cells within two cells of it (the stencil of
    the step); sides of the block that lie on the domain boundary carry the workload's kind,
    the other sides are cut off two cells away, where they cannot reach the centre update."""
    dim = w.dim
    n = w.n
    h = [(w.hi[d] - w.lo[d]) / n[d] for d in range(dim)]
    C = go.time_coefficients(dt, kappa * dt)
    out = np.zeros((fields.shape[0], len(cells)))
    strides = [1, n[0], n[0] * n[1]][:dim]
    for s, cell in enumerate(cells):
        idx = []
        rem = int(cell)
        for d in range(dim):
            idx.append(rem % n[d])
            rem //= n[d]
        lo_i = [max(idx[d] - 2, 0) for d in range(dim)]
        hi_i = [min(idx[d] + 3, n[d]) for d in range(dim)]
        shape = [hi_i[d] - lo_i[d] for d in range(dim)]
        grids = np.meshgrid(*[np.arange(lo_i[d], hi_i[d]) for d in range(dim)][::-1],
                            indexing="ij")[::-1]
        gid = sum(g.ravel() * strides[d] for d, g in enumerate(grids))
        bc = []
        for d in range(dim):
            if w.bc[2 * d] == "periodic":
                raise ValueError("block sampling needs non-periodic sides")
            bc += ["nrbc", "nrbc"]
        mesh = go.cartesian_mesh(tuple(shape), tuple(w.lo[d] + lo_i[d] * h[d] for d in range(dim)),
                                 tuple(w.lo[d] + hi_i[d] * h[d] for d in range(dim)), tuple(bc))
        V = go.fields_to_state(fields[:, gid], dim)
        m = go.material_diag(w.eps[gid], None if w.mu is None else w.mu[gid])
        jz = None
        if w.jz_mask is not None:
            jz = w.jz_mask[gid] * go.source_signal(t, *w.src)
        Vn = go.step(mesh, V, m, dt, C, c, jz)
        local = sum((idx[d] - lo_i[d]) * int(np.prod(shape[:d])) for d in range(dim))
        out[:, s] = go.state_to_fields(Vn[local:local + 1], dim)[:, 0]
    return out
