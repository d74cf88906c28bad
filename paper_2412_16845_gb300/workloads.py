"""Seeded synthetic inputs shaped like the paper's workloads.

This module only *generates inputs*: grids of material values, initial fields, source masks and
tetrahedral meshes.  It holds none of the gas-kinetic scheme's arithmetic (no fluxes, gradients,
time-integration coefficients or geometry of faces), so the CUDA library and the FP64 oracle can
both be fed from it without sharing any of the method.

Every generator draws from ``numpy.random.Generator(PCG64(SEED_BASE + config_index))`` and returns
plain float64 / int64 numpy arrays in *user cell order*: Cartesian cells are numbered with x
fastest (``i + nx*(j + ny*k)``), tetrahedra in the order they are emitted by
:func:`kuhn_tet_mesh`.  Fields are returned as ``[ncomp][ncell]`` arrays with the components
(Ez, Hx, Hy) in 2-D TM and (Ex, Ey, Ez, Hx, Hy, Hz) in 3-D.

Units follow the paper's numerical section: c = eps0 = mu0 = 1 (Sec. 5).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20241216

# Source waveform of the line-source workloads: J_z(x,t) = mask(x) * A * exp(-((t-t0)/s)^2)
# * sin(2 pi f0 (t - t0)), a Gaussian-modulated sinusoid with centre frequency f0 = 20.
SRC_A = 1.0
SRC_F0 = 20.0
SRC_S = 0.5 / SRC_F0
SRC_T0 = 3.0 * SRC_S


def rng_for(config_index: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + int(config_index)))


def cell_centres_2d(nx: int, ny: int, lo=(0.0, 0.0), hi=(1.0, 1.0)):
    """Cell-centre coordinates (x, y), each of shape [ncell], user order (x fastest)."""
    hx = (hi[0] - lo[0]) / nx
    hy = (hi[1] - lo[1]) / ny
    x = lo[0] + (np.arange(nx) + 0.5) * hx
    y = lo[1] + (np.arange(ny) + 0.5) * hy
    X, Y = np.meshgrid(x, y, indexing="xy")  # [ny][nx]
    return X.ravel(), Y.ravel()


def cell_centres_3d(nx: int, ny: int, nz: int, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
    h = [(hi[d] - lo[d]) / n for d, n in enumerate((nx, ny, nz))]
    x = lo[0] + (np.arange(nx) + 0.5) * h[0]
    y = lo[1] + (np.arange(ny) + 0.5) * h[1]
    z = lo[2] + (np.arange(nz) + 0.5) * h[2]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")  # [nz][ny][nx]
    return X.ravel(), Y.ravel(), Z.ravel()


def smoothed_noise(rng: np.random.Generator, shape, sigma_cells) -> np.ndarray:
    """Gaussian-smoothed N(0,1) noise (periodic FFT filter), min-max normalised to [0, 1].

    ``shape`` is in numpy (slowest-first) order; ``sigma_cells`` is the filter width in cells
    (one value per axis)."""
    w = rng.standard_normal(shape)
    W = np.fft.rfftn(w)
    filt = np.ones(W.shape)
    for ax, n in enumerate(shape):
        if ax == len(shape) - 1:
            k = np.fft.rfftfreq(n) * 2.0 * np.pi
        else:
            k = np.fft.fftfreq(n) * 2.0 * np.pi
        g = np.exp(-0.5 * (sigma_cells[ax] * k) ** 2)
        sh = [1] * len(shape)
        sh[ax] = g.size
        filt = filt * g.reshape(sh)
    p = np.fft.irfftn(W * filt, s=shape, axes=tuple(range(len(shape))))
    p = (p - p.min()) / (p.max() - p.min())
    return p


def plane_wave_tm(x, y, t, kvec=(2.0, 1.0)):
    """Exact TM plane wave Ez = cos(k.x - |k| t), H = Ez (sin th, -cos th) with k = 2 pi kvec.

    With th = 0 this is the paper's plane wave E_z = cos 2pi(x - ct), B_y = -E_z (Sec. 5.1).
    kvec must be integer for the wave to be periodic on the unit square."""
    k = 2.0 * np.pi * np.asarray(kvec, dtype=np.float64)
    kn = float(np.hypot(k[0], k[1]))
    th = math.atan2(k[1], k[0])
    ez = np.cos(k[0] * x + k[1] * y - kn * t)
    return np.stack([ez, math.sin(th) * ez, -math.cos(th) * ez])


def gaussian_pulse_tm_periodic(x, y, centre, sigma):
    """Ez = exp(-r^2/(2 sigma^2)) with minimum-image distance on the unit square; H = 0."""
    dx = x - centre[0]
    dy = y - centre[1]
    dx -= np.round(dx)
    dy -= np.round(dy)
    ez = np.exp(-(dx * dx + dy * dy) / (2.0 * sigma * sigma))
    z = np.zeros_like(ez)
    return np.stack([ez, z, z])


def source_waveform(t, A=SRC_A, f0=SRC_F0, t0=SRC_T0, s=SRC_S):
    """Reference copy of the line-source time signal, for tests that need it on the host."""
    return A * math.exp(-(((t - t0) / s) ** 2)) * math.sin(2.0 * math.pi * f0 * (t - t0))


@dataclass
class CartWorkload:
    """A Cartesian workload: sizes, box, boundary kinds, materials, initial fields, source."""
    name: str
    dim: int
    n: tuple
    lo: tuple
    hi: tuple
    bc: tuple                 # per side (-x,+x,-y,+y[,-z,+z]): "periodic" | "nrbc" | "pec"
    cfl: float
    steps: int
    eps: np.ndarray           # [ncell]
    mu: np.ndarray | None     # [ncell] or None (= 1)
    fields0: np.ndarray       # [ncomp][ncell]
    jz_mask: np.ndarray | None = None   # [ncell] or None
    src: tuple = (SRC_A, SRC_F0, SRC_T0, SRC_S)   # "cw": (A, f0, t0)
    waveform: str = "gauss_sine"         # "gauss_sine" or "cw" (continuous cosine)
    phm: tuple | None = None             # (chi, gamma): divergence cleaning (2-D: fields gain psi)
    probe: np.ndarray | None = None      # int64 cell ids
    design: np.ndarray | None = None     # int64 cell ids
    c_lattice: float = 1.0               # lattice speed c of the workload (c = 1 in Sec. 5)
    limiter: str | None = None           # None or "vanleer" (limited slopes)
    extra: dict = field(default_factory=dict)

    @property
    def ncell(self) -> int:
        return int(np.prod(self.n))


def config1_periodic_tm(n: int = 64, with_pulse: bool = True, kvec=(2.0, 1.0)) -> CartWorkload:
    """2-D TM, periodic unit square, vacuum, oblique plane wave + seeded Gaussian pulse, CFL 0.5.

    The nominal '30 degrees, wavelength 0.5' wave is not periodic on the unit square; the
    nearest periodic-compatible wave vector k = 2pi(2,1) (26.57 deg, wavelength 1/sqrt(5)) is
    used instead."""
    rng = rng_for(1)
    x, y = cell_centres_2d(n, n)
    f = plane_wave_tm(x, y, 0.0, kvec)
    centre = rng.uniform(0.0, 1.0, size=2)
    if with_pulse:
        f = f + gaussian_pulse_tm_periodic(x, y, centre, 0.05)
    return CartWorkload(
        name=f"tm2d_periodic_{n}", dim=2, n=(n, n), lo=(0.0, 0.0), hi=(1.0, 1.0),
        bc=("periodic",) * 4, cfl=0.5, steps=200, eps=np.ones(n * n), mu=None,
        fields0=f, extra={"pulse_centre": centre, "kvec": kvec})


def _cylinders(rng, count, rmin, rmax, box_lo, box_hi, gap, keep_clear_x=None):
    cyl = []
    tries = 0
    while len(cyl) < count:
        tries += 1
        if tries > 200000:
            raise RuntimeError("cylinder placement failed")
        c = rng.uniform(box_lo, box_hi, size=2)
        r = rng.uniform(rmin, rmax)
        e = rng.uniform(2.0, 6.0)
        if keep_clear_x is not None and abs(c[0] - keep_clear_x) < r + gap:
            continue
        if all(np.hypot(c[0] - q[0], c[1] - q[1]) >= r + q[2] + gap for q in cyl):
            cyl.append((c[0], c[1], r, e))
    return cyl


def config2_cylinders_tm(n: int = 4096, steps: int = 2000) -> CartWorkload:
    """2-D TM on [0,1]^2 with 32 seeded dielectric cylinders (r in [0.01,0.03], eps in [2,6],
    mu = 1), non-reflecting boundary on all sides, a Gaussian-modulated line source (centre
    frequency 20) on the cell column at x = 0.25, CFL 0.5.  Fields start at zero."""
    rng = rng_for(2)
    x, y = cell_centres_2d(n, n)
    h = 1.0 / n
    src_x = 0.25
    cyl = _cylinders(rng, 32, 0.01, 0.03, 0.1, 0.9, 0.005, keep_clear_x=src_x)
    eps = np.ones(n * n)
    for cx, cy, r, e in cyl:
        eps[(x - cx) ** 2 + (y - cy) ** 2 <= r * r] = e
    i_src = int(src_x * n)
    mask = np.zeros(n * n)
    mask[(np.arange(n * n) % n) == i_src] = 1.0 / h
    return CartWorkload(
        name=f"tm2d_cylinders_{n}", dim=2, n=(n, n), lo=(0.0, 0.0), hi=(1.0, 1.0),
        bc=("nrbc",) * 4, cfl=0.5, steps=steps, eps=eps, mu=None,
        fields0=np.zeros((3, n * n)), jz_mask=mask, extra={"cylinders": cyl, "i_src": i_src})


def dipole_tm(n: int = 100, two: bool = False, t_end: float | None = None,
              J0: float = 1.0, T: float = 0.1) -> CartWorkload:
    """The oscillating electric dipole of Sec. 5.4: a z-directed current J_z = J0 cos(2 pi t/T)
    on the 2 x 2 cells around the dipole point (the points are cell corners), vacuum,
    non-reflecting boundary on all sides, CFL 0.5, fields start at zero.  One dipole at the
    centre of [0,1]^2 on n x n cells (run to t = 3), or two at (0.7, 0.5) and (1.3, 0.5) on
    [0,2] x [0,1] with 2n x n cells (run to t = 2)."""
    nx, ny = (2 * n, n) if two else (n, n)
    Lx = 2.0 if two else 1.0
    h = Lx / nx
    pts = [(0.7, 0.5), (1.3, 0.5)] if two else [(0.5, 0.5)]
    mask = np.zeros(nx * ny)
    for px, py in pts:
        i, j = int(round(px / h)), int(round(py / h))      # the dipole point is the corner i, j
        for jj in (j - 1, j):
            for ii in (i - 1, i):
                mask[jj * nx + ii] = 1.0
    t_end = t_end if t_end is not None else (2.0 if two else 3.0)
    dt = 0.5 * h
    steps = int(math.ceil(t_end / dt - 1e-9))
    return CartWorkload(
        name=f"tm2d_dipole{'2' if two else ''}_{n}", dim=2, n=(nx, ny), lo=(0.0, 0.0),
        hi=(Lx, 1.0), bc=("nrbc",) * 4, cfl=0.5, steps=steps, eps=np.ones(nx * ny), mu=None,
        fields0=np.zeros((3, nx * ny)), jz_mask=mask, src=(J0, 1.0 / T, 0.0), waveform="cw",
        extra={"dipoles": pts, "t_end": t_end})


def incident_pulse_3d(x):
    """x-directed Gaussian pulse Ez = exp(-((x-0.15)/0.05)^2), Hy = -Ez, other components 0."""
    ez = np.exp(-(((x - 0.15) / 0.05) ** 2))
    z = np.zeros_like(ez)
    return np.stack([z, z, ez, z, -ez, z])


def config3_sphere_3d(n: int = 256, steps: int = 500) -> CartWorkload:
    """3-D Maxwell on the unit cube: dielectric sphere (r = 0.2, eps = 2.25) at the centre plus
    a smoothed random eps perturbation (amplitude 0.1, correlation length 0.05), incident
    x-directed pulse, non-reflecting boundary on all sides, CFL 0.4."""
    rng = rng_for(3)
    x, y, z = cell_centres_3d(n, n, n)
    p = smoothed_noise(rng, (n, n, n), (0.05 * n,) * 3).ravel()
    inside = (x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2 <= 0.2 ** 2
    eps = np.where(inside, 2.25, 1.0) + 0.1 * p
    return CartWorkload(
        name=f"maxwell3d_sphere_{n}", dim=3, n=(n, n, n), lo=(0.0,) * 3, hi=(1.0,) * 3,
        bc=("nrbc",) * 6, cfl=0.4, steps=steps, eps=eps, mu=None, fields0=incident_pulse_3d(x))


def config5_design_tm(n: int = 2048, steps: int = 2000) -> CartWorkload:
    """2-D TM inverse-design workload: line source on the left (x = 0.30), a design square
    x in [0.3125, 0.5625], y in [0.375, 0.625] whose eps is Gaussian-smoothed noise mapped to
    [1, 4], a probe disc of radius 0.02 at (0.5, 0.5), non-reflecting boundary, CFL 0.5."""
    rng = rng_for(5)
    x, y = cell_centres_2d(n, n)
    h = 1.0 / n
    i0, i1 = int(round(0.3125 * n)), int(round(0.5625 * n))
    j0, j1 = int(round(0.375 * n)), int(round(0.625 * n))
    nd_x, nd_y = i1 - i0, j1 - j0
    p = smoothed_noise(rng, (nd_y, nd_x), (0.01 * n, 0.01 * n))
    eps = np.ones(n * n)
    ii = np.arange(i0, i1)
    jj = np.arange(j0, j1)
    design = (jj[:, None] * n + ii[None, :]).ravel().astype(np.int64)
    eps[design] = 1.0 + 3.0 * p.ravel()
    probe = np.nonzero((x - 0.5) ** 2 + (y - 0.5) ** 2 <= 0.02 ** 2)[0].astype(np.int64)
    i_src = int(0.30 * n)
    mask = np.zeros(n * n)
    mask[(np.arange(n * n) % n) == i_src] = 1.0 / h
    return CartWorkload(
        name=f"tm2d_design_{n}", dim=2, n=(n, n), lo=(0.0, 0.0), hi=(1.0, 1.0),
        bc=("nrbc",) * 4, cfl=0.5, steps=steps, eps=eps, mu=None,
        fields0=np.zeros((3, n * n)), jz_mask=mask, probe=probe, design=design,
        extra={"design_box": (i0, i1, j0, j1), "i_src": i_src})


# --------------------------------------------------------------------------------------------
# Tetrahedral meshes
# --------------------------------------------------------------------------------------------

@dataclass
class TetWorkload:
    name: str
    vert: np.ndarray      # [nvert][3] float64
    tet: np.ndarray       # [ntet][4] int64, positively oriented
    cfl: float
    steps: int
    eps: np.ndarray       # [ntet]
    mu: np.ndarray | None
    fields0: np.ndarray   # [6][ntet]
    extra: dict = field(default_factory=dict)

    @property
    def ncell(self) -> int:
        return int(self.tet.shape[0])


# The six Kuhn (Freudenthal) tetrahedra of a unit hex: one per permutation of the axes, all
# sharing the diagonal from corner (0,0,0) to corner (1,1,1).  Neighbouring hexes split this way
# match face to face.
_KUHN_PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


def kuhn_tet_mesh(m: int, jitter: float, rng: np.random.Generator | None):
    """Unit cube split into m^3 hexes, each into the 6 Kuhn tetrahedra.

    Interior vertices are moved by independent uniform offsets in [-jitter*h, jitter*h] per
    coordinate (boundary vertices stay on the cube faces).  Returns (vert [nv][3], tet [nt][4])
    with every tetrahedron positively oriented."""
    h = 1.0 / m
    nv1 = m + 1
    g = np.arange(nv1)
    K, J, I = np.meshgrid(g, g, g, indexing="ij")
    vert = np.stack([I.ravel() * h, J.ravel() * h, K.ravel() * h], axis=1).astype(np.float64)
    if jitter > 0.0:
        interior = ((I > 0) & (I < m) & (J > 0) & (J < m) & (K > 0) & (K < m)).ravel()
        off = rng.uniform(-jitter * h, jitter * h, size=(vert.shape[0], 3))
        vert[interior] += off[interior]

    def vid(i, j, k):
        return i + nv1 * (j + nv1 * k)

    hk, hj, hi = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    hi = hi.ravel(); hj = hj.ravel(); hk = hk.ravel()
    tets = []
    for perm in _KUHN_PERMS:
        cur = np.stack([hi, hj, hk], axis=1).copy()
        ids = [vid(cur[:, 0], cur[:, 1], cur[:, 2])]
        for ax in perm:
            cur[:, ax] += 1
            ids.append(vid(cur[:, 0], cur[:, 1], cur[:, 2]))
        tets.append(np.stack(ids, axis=1))
    tet = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int64)   # hex-major, 6 per hex
    # orient positively
    p = vert[tet]
    d = np.einsum("ij,ij->i", np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), p[:, 3] - p[:, 0])
    neg = d < 0
    tet[neg, 2], tet[neg, 3] = tet[neg, 3].copy(), tet[neg, 2].copy()
    return vert, tet


def config4_tets(m: int = 64, steps: int = 500, jitter: float = 0.1) -> TetWorkload:
    """Unstructured tetrahedral workload: m^3 hexes x 6 Kuhn tets, interior vertices jittered by
    +-0.1h, eps = 4 inside a centred sphere of radius 0.25 (by tet centroid), 1 outside,
    non-reflecting outer boundary, incident x-directed pulse, CFL 0.4."""
    rng = rng_for(4)
    vert, tet = kuhn_tet_mesh(m, jitter, rng)
    cen = vert[tet].mean(axis=1)
    r2 = ((cen - 0.5) ** 2).sum(axis=1)
    eps = np.where(r2 <= 0.25 ** 2, 4.0, 1.0)
    return TetWorkload(name=f"tets_sphere_{m}", vert=vert, tet=tet, cfl=0.4, steps=steps,
                       eps=eps, mu=None, fields0=incident_pulse_3d(cen[:, 0]),
                       extra={"m": m})


def riemann_3d(n: int = 200, t_end: float = 0.25, limiter: str | None = "vanleer") -> CartWorkload:
    """The electromagnetic Riemann problem of Sec. 5.3 on a 3-D grid: left state E_y = 1,
    B_x = 1, B_y = -0.75 and right state E_y = -1, B_x = 1, B_y = 0.75 (all else 0), jump at
    x = 0.5, t_end = 0.25, CFL 0.5, cell size 0.01 as in the paper (n = 200).  The x extent is
    [-0.5, 1.5] with non-reflecting ends, so that the waves the kinetic boundary sends in from
    the non-zero end states (speed 1) stay outside [0, 1] until t = 0.5; y and z are periodic and
    two cells deep (the problem is 1-D).  H = B (c = 1)."""
    h = 2.0 / n
    idx = np.arange(n * 4)
    x = -0.5 + (idx % n + 0.5) * h
    left = x < 0.5
    f = np.zeros((6, idx.size))
    f[1] = np.where(left, 1.0, -1.0)
    f[3] = 1.0
    f[4] = np.where(left, -0.75, 0.75)
    return CartWorkload(
        name=f"riemann3d_{n}", dim=3, n=(n, 2, 2), lo=(-0.5, 0.0, 0.0), hi=(1.5, 2 * h, 2 * h),
        bc=("nrbc", "nrbc") + ("periodic",) * 4, cfl=0.5, steps=0, eps=np.ones(idx.size),
        mu=None, fields0=f, limiter=limiter, extra={"t_end": t_end, "x": x})
