"""The FP32 tet path reads its geometry (face normals and the frame's 1/(1 + n_1), from which
the kernel forms the frame rows in FP32; face-centroid offsets, areas, face weights, update
weights) rounded to FP32 once on the host.  This measures what that rounding alone does
to the method: the FP64 oracle run on the jittered Kuhn-tet sphere workload with every
geometric quantity rounded to FP32 (same dt, computed from the FP64 geometry as the library
does) stays within 1e-6 relative L2 of the run on the FP64 geometry after 30 steps (measured
1.5e-7), two orders of magnitude below the FP32 parity tolerance (2e-5) that the FP32 fields
are held to."""
import dataclasses

import numpy as np

from oracle import gks_oracle as go
from paper_2412_16845_gb300 import workloads as wl


def test_fp32_geometry_changes_the_oracle_by_under_1e_6():
    w = wl.config4_tets(m=6, steps=30)
    mesh = go.tet_mesh(w.vert, w.tet)

    def r32(a):
        return a.astype(np.float32).astype(np.float64)

    mesh32 = dataclasses.replace(mesh, vol=r32(mesh.vol), centroid=r32(mesh.centroid),
                                 normal=r32(mesh.normal), area=r32(mesh.area), dL=r32(mesh.dL),
                                 dR=r32(mesh.dR))
    dt = go.time_step(mesh, w.cfl)
    ref, _ = go.run(mesh, w.fields0, w.eps, None, w.cfl, 30, dt=dt)
    rounded, _ = go.run(mesh32, w.fields0, w.eps, None, w.cfl, 30, dt=dt)
    d = np.linalg.norm(rounded - ref) / np.linalg.norm(ref)
    assert 0.0 < d <= 1e-6, d
