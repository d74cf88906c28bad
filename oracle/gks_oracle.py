"""FP64 CPU oracle of the discrete-velocity gas-kinetic scheme (GKS) for Maxwell's equations.

TEST INFRASTRUCTURE ONLY.  This module is the slow, literal statement of the scheme that the
CUDA library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The product path never
calls it, and it shares no code, tables or helpers with the CUDA path.

What it computes (paper: Pu, Long & Xu, "A Gas-Kinetic Scheme for Maxwell Equations",
arXiv 2412.16845), in the paper's order and notation:

* Sec. 2.1: the flux functions F_j(U) = A_j U of the Maxwell system, and of the
  divergence-cleaning (PHM) system with potentials phi, psi and speeds chi, gamma.
* Sec. 2.2: the D3Q4 lattice (D2Q4 in 2-D) and the local equilibrium
  g_k = U/4 + F(U).u_k / (4 c^2), with the compatibility constraints sum g = U, sum u^j g = F_j.
* Sec. 3.1: the finite-volume update U^{n+1} = U^n - dt/|Omega| sum |l_s| F_s + dt S^n, the
  local-frame rotation T = diag(T', T'), the interface equilibrium
  <g0> = <g^l>_{>0} + <g^r>_{<0} and its gradient, the Green-Gauss cell gradient, the time
  derivative from <g_t + u.grad g0> = 0, and the time-integrated flux with C1..C5.
* Sec. 3.1 (last paragraph): the kinetic non-reflecting boundary (incoming distributions of the
  ghost cell are zero).
* Sec. 5.5: perfect-electric-conductor walls (mirror ghosts); Sec. 5.4: the time-harmonic dipole
  current; Sec. 5.3: limited slopes (van Leer, a reading).

Every step is written per discrete velocity, exactly as the paper states it; no closed form of
the flux is used here (the tests derive the closed forms independently and compare).

Readings of passages that are silent, garbled or ambiguous:

* Materials (the paper has none): V = (E, H) is stored, U = M V with M = diag(eps I, mu I);
  F_j acts on V exactly like the paper's F_j acts on (E, c^2 B); the interface equilibrium uses
  M_s = (M_L + M_R)/2 (M_L on a boundary face).  With eps = mu = 1 this is the paper's scheme.
* c_4 = e^{-t/tau}, c_5 = t e^{-t/tau} (the printed positive exponents are a sign slip; the
  printed closed forms of C_4, C_5 already carry e^{-dt/tau}).
* Upwind sets: l for u_k.n > 0, r for u_k.n < 0 (u_k.n never vanishes in the local frame).
* "U_k/4" in the equilibrium is U/4.
* tau = kappa * dt with kappa a parameter; kappa = 0 means the tau -> 0 limit coefficients
  (Sec. 4.1, non-viscous limit): C1 = dt, C3 = dt^2/2, C2 = C4 = C5 = 0.
* Ghost values for Green-Gauss at a non-reflecting face: a copy of the interior cell.
* Limiter (Sec. 5.3 names none): van Leer's, on the one-sided differences of each component of
  V along each axis of a Cartesian grid (limited_gradient); off unless asked for.
* Face orientation: Cartesian faces use n = +e_d with L the cell on the -e_d side (wrap faces
  included); tetrahedral interior faces point from the smaller to the larger user cell index;
  boundary faces point outward.
* Source: S = (-J, 0) with J evaluated at t^n (explicit).
* Time step: dt = CFL * h_min / c with h_i = 2 dim |Omega_i| / sum_s |l_s| (= the edge of a
  square or cube).

Units: c = eps0 = mu0 = 1 (Sec. 5) unless a lattice speed c is passed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# --------------------------------------------------------------------------------------------
# Sec. 2.1 -- flux functions F_j(U) = A_j U with chi = gamma = 0
# --------------------------------------------------------------------------------------------

# The 3x3 blocks M_1, M_2, M_3 of the flux Jacobians, as printed in Sec. 2.1.
M_BLOCKS = np.array([
    [[0, 0, 0], [0, 0, 1], [0, -1, 0]],
    [[0, 0, -1], [0, 0, 0], [1, 0, 0]],
    [[0, 1, 0], [-1, 0, 0], [0, 0, 0]],
], dtype=np.float64)


def flux_dir(j: int, V, phm=None):
    """F_j(V) for direction j in {0,1,2}: the E rows are M_j H, the B (here H) rows M_j^T E.

    V has shape [..., 6] = (E, H), or [..., 8] = (E, H, phi, psi) for the divergence-cleaning
    (PHM) system with phm = (chi, gamma): then E_j gains chi phi, H_j gains gamma psi, and the
    phi and psi rows are chi E_j and gamma H_j.  In the paper's units H = c^2 B (c = 1), so this
    is the printed F_j(U) of Sec. 2.1."""
    Mj = M_BLOCKS[j]
    out = np.zeros(V.shape, dtype=V.dtype)
    out[..., 0:3] = V[..., 3:6] @ Mj.T      # M_j H
    out[..., 3:6] = V[..., 0:3] @ Mj        # M_j^T E
    if V.shape[-1] == 8:
        chi, gamma = phm if phm is not None else (0.0, 0.0)
        out[..., j] = out[..., j] + chi * V[..., 6]
        out[..., 3 + j] = out[..., 3 + j] + gamma * V[..., 7]
        out[..., 6] = chi * V[..., j]
        out[..., 7] = gamma * V[..., 3 + j]
    return out


# --------------------------------------------------------------------------------------------
# Sec. 2.2 -- lattice and local equilibrium
# --------------------------------------------------------------------------------------------

def lattice(dim: int, c: float = 1.0) -> np.ndarray:
    """Discrete velocities u_k, shape [4, 3].

    3-D: the D3Q4 set c(1,1,1), c(1,-1,-1), c(-1,1,-1), c(-1,-1,1) (Sec. 2.2).
    2-D: the same set projected on the (x, y) plane, i.e. D2Q4 = c(+-1, +-1, 0)."""
    u = c * np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64)
    if dim == 2:
        u[:, 2] = 0.0
    return u


def equilibrium(U, V, uk, c: float, phm=None):
    """g_k = U/4 + sum_j u_k^j F_j(V) / (4 c^2)  (Sec. 2.2; material reading U = M V)."""
    g = U / 4.0
    for j in range(3):
        if uk[j] != 0.0:
            g = g + uk[j] * flux_dir(j, V, phm) / (4.0 * c * c)
    return g


def equilibria(U, V, u, c: float, phm=None):
    """[g_0, g_1, g_2, g_3] for all four lattice velocities (the same formula as
    :func:`equilibrium`, with the three F_j(V) evaluated once)."""
    F = [flux_dir(j, V, phm) for j in range(3)]
    out = []
    for k in range(u.shape[0]):
        g = U / 4.0
        for j in range(3):
            if u[k, j] != 0.0:
                g = g + u[k, j] * F[j] / (4.0 * c * c)
        out.append(g)
    return out


# --------------------------------------------------------------------------------------------
# Sec. 3.1 -- time-integration coefficients C1..C5
# --------------------------------------------------------------------------------------------

def time_coefficients(dt: float, tau: float):
    """C1..C5 = integrals over [0, dt] of c1..c5 (Sec. 3.1), with c4 = e^{-t/tau},
    c5 = t e^{-t/tau}.

    tau = 0 gives the non-viscous limit (Sec. 4.1): (dt, 0, dt^2/2, 0, 0).  For x = dt/tau < 2
    the closed forms lose digits to cancellation, so their Taylor series in x (derived from the
    same closed forms) are summed instead."""
    if tau == 0.0:
        return (dt, 0.0, 0.5 * dt * dt, 0.0, 0.0)
    x = dt / tau
    if x >= 2.0:
        E = math.exp(-x)
        ome = -math.expm1(-x)                      # 1 - e^{-dt/tau}
        C1 = dt - tau * ome
        C2 = tau * (-dt + 2.0 * tau * ome - dt * E)
        C3 = 0.5 * dt * dt - tau * dt + tau * tau * ome
        C4 = tau * ome
        C5 = -tau * dt * E + tau * tau * ome
        return (C1, C2, C3, C4, C5)
    # series: with s_n = (-1)^n x^(n-2) / n!
    c1 = c2 = c3 = c4 = c5 = 0.0
    fact = 1.0
    for n in range(1, 60):
        fact *= n
        sgn = -1.0 if n % 2 else 1.0
        c4 += -sgn * x ** (n - 1) / fact               # (1-E)/x
        if n >= 2:
            c1 += sgn * x ** (n - 1) / fact            # 1 - (1-E)/x
            c5 += sgn * (n - 1) * x ** (n - 2) / fact  # [(1-E) - xE]/x^2
        if n >= 3:
            c3 += -sgn * x ** (n - 2) / fact           # 1/2 - 1/x + (1-E)/x^2
            c2 += sgn * (n - 2) * x ** (n - 2) / fact  # [-x + 2(1-E) - xE]/x^2
    return (dt * c1, dt * dt * c2, dt * dt * c3, dt * c4, dt * dt * c5)


# --------------------------------------------------------------------------------------------
# Sec. 3.1 -- rotation into the face frame
# --------------------------------------------------------------------------------------------

def rotation(n) -> np.ndarray:
    """T'(n) of Sec. 3.1 for unit normals n [nf, 3] -> [nf, 3, 3].

    Row 1 is n itself.  n_1 = -1 uses the printed special case diag(-1, -1, 1).  1 + n_1 is
    evaluated as (n_2^2 + n_3^2)/(1 - n_1) when n_1 < 0 (equal for a unit n, without the
    cancellation near n_1 = -1)."""
    n = np.asarray(n, dtype=np.float64)
    n1, n2, n3 = n[:, 0], n[:, 1], n[:, 2]
    special = n1 == -1.0
    den = np.where(n1 >= 0.0, 1.0, 1.0 - n1)
    one_p = np.where(n1 >= 0.0, 1.0 + n1, (n2 * n2 + n3 * n3) / den)
    inv = 1.0 / np.where(special, 1.0, one_p)
    T = np.empty((n.shape[0], 3, 3))
    T[:, 0, 0], T[:, 0, 1], T[:, 0, 2] = n1, n2, n3
    T[:, 1, 0], T[:, 1, 1], T[:, 1, 2] = -n2, n1 + n3 * n3 * inv, -n2 * n3 * inv
    T[:, 2, 0], T[:, 2, 1], T[:, 2, 2] = -n3, -n2 * n3 * inv, 1.0 - n3 * n3 * inv
    T[special] = np.diag([-1.0, -1.0, 1.0])
    return T


def _rot_vec6(T, V):
    """Apply diag(T', T') to [nf, 6] vectors (the scalars phi, psi of [nf, 8] stay)."""
    out = V.copy()
    V3 = V[:, :6].reshape(V.shape[0], 2, 3)
    out[:, :6] = np.matmul(V3, np.swapaxes(T, 1, 2)).reshape(V.shape[0], 6)   # (T' v)^T = v^T T'^T
    return out


def _rot_vec6_back(T, V):
    """Apply diag(T', T')^{-1} = diag(T'^T, T'^T) (scalars unchanged)."""
    out = V.copy()
    V3 = V[:, :6].reshape(V.shape[0], 2, 3)
    out[:, :6] = np.matmul(V3, T).reshape(V.shape[0], 6)
    return out


def _rot_grad(T, G):
    """Rotate gradients G [nf, 3(direction), ncomp(field)]: field index by T (the E and H
    3-vectors), direction by T'."""
    nf = G.shape[0]
    G2 = G.copy()
    G3 = G[:, :, :6].reshape(nf, 6, 3)             # rows (direction, block), columns component
    G3 = np.matmul(G3, np.swapaxes(T, 1, 2))       # field components: T' applied to each 3-vector
    G2[:, :, :6] = G3.reshape(nf, 3, 6)
    return np.matmul(T, G2)                        # direction index: d'_a = sum_d T'[a, d] d_d


# --------------------------------------------------------------------------------------------
# Sec. 3.1 -- the GKS interface flux, literally per discrete velocity
# --------------------------------------------------------------------------------------------

def face_flux_local(Vl, Gl, ml, Vr, Gr, mr, ghost, C, dt, c, dim, phm=None):
    """Time-averaged numerical flux in the face frame (normal = local x).

    Vl, Vr [nf, 6]: reconstructed primitive states (E, H) on the two sides ([nf, 8] with the
    cleaning potentials phi, psi when phm = (chi, gamma) is given).
    Gl, Gr [nf, 3, 6]: their gradients, Gl[:, j] = d/dx_j V^l.
    ml, mr [nf, 6]: diagonals of M on each side.
    ghost [nf] bool: kinetic non-reflecting face -- the r side is a ghost cell whose
    distributions are all zero (its incoming half is what enters the interface).
    Returns F~ [nf, 6] = (1/dt)[C1<u g0> + C2<u u.grad g0> + C3<u g_t>
                               + C4(<u g^l>_{>0} + <u g^r>_{<0})
                               - C5(<u u.grad g^l>_{>0} + <u u.grad g^r>_{<0})]."""
    C1, C2, C3, C4, C5 = C
    u = lattice(dim, c)
    keep_r = (~ghost).astype(np.float64)[:, None]
    Ul, Ur = ml * Vl, mr * Vr

    gl = equilibria(Ul, Vl, u, c, phm)
    gr = [keep_r * g for g in equilibria(Ur, Vr, u, c, phm)]
    dgl_j = [equilibria(ml * Gl[:, j], Gl[:, j], u, c, phm) for j in range(3)]
    dgr_j = [[keep_r * g for g in equilibria(mr * Gr[:, j], Gr[:, j], u, c, phm)] for j in range(3)]
    dgl = [[dgl_j[j][k] for j in range(3)] for k in range(4)]      # dgl[k][j] = d_j g_k^l
    dgr = [[dgr_j[j][k] for j in range(3)] for k in range(4)]
    pos = [k for k in range(4) if u[k, 0] > 0.0]
    neg = [k for k in range(4) if u[k, 0] < 0.0]

    # interface equilibrium <g0> = <g^l>_{>0} + <g^r>_{<0}, and its gradient
    W0 = sum(gl[k] for k in pos) + sum(gr[k] for k in neg)
    dW0 = [sum(dgl[k][j] for k in pos) + sum(dgr[k][j] for k in neg) for j in range(3)]

    ms = np.where(ghost[:, None], ml, 0.5 * (ml + mr))
    V0 = W0 / ms
    dV0 = [dW0[j] / ms for j in range(3)]
    g0 = equilibria(W0, V0, u, c, phm)
    dg0_j = [equilibria(dW0[j], dV0[j], u, c, phm) for j in range(3)]
    dg0 = [[dg0_j[j][k] for j in range(3)] for k in range(4)]

    # compatibility: <g_t> = -<u . grad g0>; g_t is the equilibrium of that moment
    W0t = -sum(u[k, j] * dg0[k][j] for k in range(4) for j in range(3))
    gt = equilibria(W0t, W0t / ms, u, c, phm)

    def u_dot_grad(dg, k):
        return sum(u[k, j] * dg[k][j] for j in range(3))

    T1 = sum(u[k, 0] * g0[k] for k in range(4))
    T2 = sum(u[k, 0] * u_dot_grad(dg0, k) for k in range(4))
    T3 = sum(u[k, 0] * gt[k] for k in range(4))
    T4 = sum(u[k, 0] * gl[k] for k in pos) + sum(u[k, 0] * gr[k] for k in neg)
    T5 = sum(u[k, 0] * u_dot_grad(dgl, k) for k in pos) + \
        sum(u[k, 0] * u_dot_grad(dgr, k) for k in neg)
    return (C1 * T1 + C2 * T2 + C3 * T3 + C4 * T4 - C5 * T5) / dt


# --------------------------------------------------------------------------------------------
# Finite-volume meshes (Sec. 3.1): cell volumes, face areas, normals, offsets
# --------------------------------------------------------------------------------------------

@dataclass
class FVMesh:
    dim: int
    vol: np.ndarray        # [ncell]
    centroid: np.ndarray   # [ncell, 3]
    L: np.ndarray          # [nface] int64
    R: np.ndarray          # [nface] int64, -1 on boundary faces
    normal: np.ndarray     # [nface, 3] unit, L -> R (boundary: outward)
    area: np.ndarray       # [nface]
    dL: np.ndarray         # [nface, 3] x_s - x_L
    dR: np.ndarray         # [nface, 3] x_s - x_R (periodic faces use the image of R)
    boundary: np.ndarray   # [nface] bool: kinetic non-reflecting face
    pec: np.ndarray = None  # [nface] bool: perfect-electric-conductor wall (mirror ghost)

    def pec_faces(self) -> np.ndarray:
        return np.zeros(self.nface, dtype=bool) if self.pec is None else self.pec

    @property
    def ncell(self) -> int:
        return int(self.vol.shape[0])

    @property
    def nface(self) -> int:
        return int(self.L.shape[0])


def cartesian_mesh(n, lo, hi, bc) -> FVMesh:
    """Uniform Cartesian grid (2-D or 3-D), cells numbered x fastest.

    bc: per side (-x, +x, -y, +y[, -z, +z]) 'periodic', 'nrbc' (kinetic non-reflecting) or
    'pec' (perfect electric conductor).  2-D cells have unit depth in z: |Omega| = hx hy,
    |l| = edge length."""
    dim = len(n)
    n = tuple(int(v) for v in n)
    h = [(hi[d] - lo[d]) / n[d] for d in range(dim)]
    ncell = int(np.prod(n))
    idx = np.arange(ncell).reshape(n[::-1])         # [nz][ny][nx] or [ny][nx]
    coords = np.meshgrid(*[lo[d] + (np.arange(n[d]) + 0.5) * h[d] for d in range(dim)][::-1],
                         indexing="ij")[::-1]        # x, y(, z) each shaped like idx
    centroid = np.zeros((ncell, 3))
    for d in range(dim):
        centroid[:, d] = coords[d].ravel()
    vol = np.full(ncell, float(np.prod(h)))
    Ls, Rs, ns, As, dLs, dRs, bs, ps = [], [], [], [], [], [], [], []
    for d in range(dim):
        ax = dim - 1 - d                             # numpy axis of direction d
        area = float(np.prod([h[e] for e in range(dim) if e != d]))
        e = np.zeros(3)
        e[d] = 1.0
        lower = np.take(idx, np.arange(n[d] - 1), axis=ax).ravel()
        upper = np.take(idx, np.arange(1, n[d]), axis=ax).ravel()
        periodic = bc[2 * d] == "periodic"
        if periodic != (bc[2 * d + 1] == "periodic"):
            raise ValueError("periodic sides must be paired")
        first = np.take(idx, 0, axis=ax).ravel()
        last = np.take(idx, n[d] - 1, axis=ax).ravel()
        if periodic:
            lower = np.concatenate([lower, last])
            upper = np.concatenate([upper, first])
        nf = lower.size
        Ls.append(lower); Rs.append(upper)
        ns.append(np.tile(e, (nf, 1))); As.append(np.full(nf, area))
        dLs.append(np.tile(0.5 * h[d] * e, (nf, 1))); dRs.append(np.tile(-0.5 * h[d] * e, (nf, 1)))
        bs.append(np.zeros(nf, dtype=bool)); ps.append(np.zeros(nf, dtype=bool))
        if not periodic:
            for cells, sgn, side in ((first, -1.0, bc[2 * d]), (last, 1.0, bc[2 * d + 1])):
                if side not in ("nrbc", "pec"):
                    raise ValueError(f"unknown boundary {side!r}")
                nb = cells.size
                Ls.append(cells); Rs.append(np.full(nb, -1))
                ns.append(np.tile(sgn * e, (nb, 1))); As.append(np.full(nb, area))
                dLs.append(np.tile(sgn * 0.5 * h[d] * e, (nb, 1)))
                dRs.append(np.zeros((nb, 3)))
                bs.append(np.full(nb, side == "nrbc")); ps.append(np.full(nb, side == "pec"))
    return FVMesh(dim=dim, vol=vol, centroid=centroid,
                  L=np.concatenate(Ls).astype(np.int64), R=np.concatenate(Rs).astype(np.int64),
                  normal=np.concatenate(ns), area=np.concatenate(As),
                  dL=np.concatenate(dLs), dR=np.concatenate(dRs),
                  boundary=np.concatenate(bs), pec=np.concatenate(ps))


def tet_mesh(vert, tet, bc="nrbc") -> FVMesh:
    """Face-based mesh of a conforming tetrahedral mesh.

    Faces are matched on their sorted vertex triples; an interior face's normal points from the
    smaller to the larger tet index; a face seen once is a boundary face with outward normal,
    kinetic non-reflecting (bc="nrbc") or a PEC wall (bc="pec")."""
    vert = np.asarray(vert, dtype=np.float64)
    tet = np.asarray(tet, dtype=np.int64)
    nt = tet.shape[0]
    P = vert[tet]                                     # [nt, 4, 3]
    centroid = P.mean(axis=1)
    vol = np.abs(np.einsum("ij,ij->i", np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]),
                           P[:, 3] - P[:, 0])) / 6.0
    opp = [(1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2)]
    tri = np.concatenate([tet[:, list(o)] for o in opp], axis=0)      # [4 nt, 3]
    owner = np.tile(np.arange(nt), 4)
    key = np.sort(tri, axis=1)
    order = np.lexsort((key[:, 2], key[:, 1], key[:, 0]))
    ks = key[order]
    same_next = np.all(ks[1:] == ks[:-1], axis=1)
    m = ks.shape[0]
    # pair consecutive equal keys (vectorised)
    is_pair_start = np.zeros(m, dtype=bool)
    is_pair_start[:-1] = same_next
    # a key can appear at most twice in a conforming mesh
    if np.any(same_next[1:] & same_next[:-1]):
        raise ValueError("a face is shared by more than two tets")
    starts = np.nonzero(is_pair_start)[0]
    paired = np.zeros(m, dtype=bool)
    paired[starts] = True
    paired[starts + 1] = True
    a = owner[order[starts]]
    b = owner[order[starts + 1]]
    L_int = np.minimum(a, b)
    R_int = np.maximum(a, b)
    tri_int = key[order[starts]]
    single = np.nonzero(~paired)[0]
    L_bnd = owner[order[single]]
    tri_bnd = key[order[single]]
    L = np.concatenate([L_int, L_bnd])
    R = np.concatenate([R_int, np.full(L_bnd.size, -1)])
    T = np.concatenate([tri_int, tri_bnd])
    Q = vert[T]                                       # [nf, 3, 3]
    cr = np.cross(Q[:, 1] - Q[:, 0], Q[:, 2] - Q[:, 0])
    area = 0.5 * np.linalg.norm(cr, axis=1)
    nrm = cr / (2.0 * area)[:, None]
    xs = Q.mean(axis=1)
    flip = np.einsum("ij,ij->i", nrm, xs - centroid[L]) < 0.0
    nrm[flip] *= -1.0
    dL = xs - centroid[L]
    dR = np.where((R >= 0)[:, None], xs - centroid[np.maximum(R, 0)], 0.0)
    if bc not in ("nrbc", "pec"):
        raise ValueError(f"unknown boundary {bc!r}")
    return FVMesh(dim=3, vol=vol, centroid=centroid, L=L.astype(np.int64),
                  R=R.astype(np.int64), normal=nrm, area=area, dL=dL, dR=dR,
                  boundary=(R < 0) & (bc == "nrbc"), pec=(R < 0) & (bc == "pec"))


def time_step(mesh: FVMesh, cfl: float, c: float = 1.0) -> float:
    """dt = CFL h_min / c with h_i = 2 dim |Omega_i| / sum_s |l_s|."""
    perim = np.bincount(mesh.L, weights=mesh.area, minlength=mesh.ncell)
    interior = mesh.R >= 0
    perim += np.bincount(mesh.R[interior], weights=mesh.area[interior], minlength=mesh.ncell)
    h = 2.0 * mesh.dim * mesh.vol / perim
    return float(cfl * h.min() / c)


# --------------------------------------------------------------------------------------------
# Cell gradients, reconstruction, one step
# --------------------------------------------------------------------------------------------

def _scatter_add(n, idx, vals):
    """out[idx[f]] += vals[f] for vals of shape [nf, ...] (complex-safe)."""
    out = np.zeros((n,) + vals.shape[1:], dtype=vals.dtype)
    np.add.at(out, idx, vals)
    return out


def pec_mirror(n, X):
    """The field of the mirror ghost across a perfect-electric-conductor wall with unit normal n
    (Sec. 5.5 interface conditions): tangential E and normal B (H) change sign, normal E and
    tangential H are kept (their normal derivatives vanish at the wall).  X [..., 6] global
    components (E, H), n [..., 3].  With the cleaning potentials (X [..., 8]) the mirror keeps
    the parities their equations impose: phi (driven by div E, normal E even) is odd, psi
    (driven by div B, normal B odd) is even."""
    E, H = X[..., :3], X[..., 3:6]
    En = np.sum(E * n, axis=-1, keepdims=True)
    Hn = np.sum(H * n, axis=-1, keepdims=True)
    parts = [-E + 2.0 * En * n, H - 2.0 * Hn * n]
    if X.shape[-1] == 8:
        parts += [-X[..., 6:7], X[..., 7:8]]
    return np.concatenate(parts, axis=-1)


def pec_mirror_grad(n, G):
    """Gradient of the mirror ghost at the wall: the field mirror on the component index and the
    reflection I - 2 n n^T on the derivative index.  G [nf, 3, 6] (derivative, component)."""
    PG = pec_mirror(n[:, None, :], G)
    return PG - 2.0 * n[:, :, None] * np.einsum("fk,fkc->fc", n, PG)[:, None, :]


def green_gauss(mesh: FVMesh, V):
    """Cell gradients grad V_i = (1/|Omega_i|) sum_s V_s n_s |l_s|, V_s = (V_i + V_nb)/2
    (Sec. 3.1, Green-Gauss); a non-reflecting face uses a ghost equal to V_i, i.e. V_s = V_i; a
    PEC face uses the mirror ghost, V_s = (V_i + P V_i)/2.  Returns [ncell, 3, 6]."""
    inter = mesh.R >= 0
    Vs = np.where(inter[:, None], 0.5 * (V[mesh.L] + V[np.maximum(mesh.R, 0)]), V[mesh.L])
    pec = mesh.pec_faces()
    if pec.any():
        VL = V[mesh.L[pec]]
        Vs[pec] = 0.5 * (VL + pec_mirror(mesh.normal[pec], VL))
    contrib = Vs[:, None, :] * (mesh.normal * mesh.area[:, None])[:, :, None]   # [nf, 3, 6]
    G = _scatter_add(mesh.ncell, mesh.L, contrib)
    G -= _scatter_add(mesh.ncell, mesh.R[inter], contrib[inter])
    return G / mesh.vol[:, None, None]


def van_leer(a, b):
    """van Leer's limiter of two one-sided slopes: their harmonic mean 2ab/(a + b) where they
    have the same sign, 0 where they differ or one vanishes (an extremum)."""
    ab = a * b
    same = ab > 0.0
    return np.where(same, 2.0 * ab / np.where(same, a + b, 1.0), 0.0)


def limited_gradient(mesh: FVMesh, V):
    """Limited cell gradients on a Cartesian grid, [ncell, 3, ncomp].

    Reading (Sec. 5.3 uses a limiter that drops to first order at discontinuities and keeps
    second order in smooth regions, without naming it): along each axis d the slope is
    van_leer(D+, D-) of the one-sided differences D+ = (V_{i+e_d} - V_i)/h_d and
    D- = (V_i - V_{i-e_d})/h_d, per component of V, with the ghosts of the Green-Gauss gradient
    (a copy of the cell at a non-reflecting side, the mirror image at a PEC wall, the wrapped
    cell on periodic sides).  (D+ + D-)/2 is the unlimited Green-Gauss gradient."""
    axis = np.argmax(np.abs(mesh.normal), axis=1)
    if not np.allclose(np.abs(mesh.normal[np.arange(mesh.nface), axis]), 1.0):
        raise ValueError("the limiter is defined on Cartesian grids")
    h = 2.0 * np.abs(mesh.dL[np.arange(mesh.nface), axis])
    ncomp = V.shape[1]
    fwd = np.zeros((mesh.ncell, 3, ncomp), dtype=V.dtype)
    bwd = np.zeros_like(fwd)
    inter = mesh.R >= 0
    # interior face (normal +e_d, L below R): forward difference of L, backward difference of R
    fi = np.nonzero(inter)[0]
    D = (V[mesh.R[fi]] - V[mesh.L[fi]]) / h[fi, None]
    fwd[mesh.L[fi], axis[fi]] = D
    bwd[mesh.R[fi], axis[fi]] = D
    # boundary face (outward normal +-e_d): the ghost beyond the cell
    fb = np.nonzero(~inter)[0]
    VL = V[mesh.L[fb]]
    ghost = VL.copy()
    pec = mesh.pec_faces()[fb]
    if pec.any():
        ghost[pec] = pec_mirror(mesh.normal[fb][pec], VL[pec])
    up = mesh.normal[fb, axis[fb]] > 0
    Db = (ghost - VL) / h[fb, None]
    fwd[mesh.L[fb[up]], axis[fb[up]]] = Db[up]
    bwd[mesh.L[fb[~up]], axis[fb[~up]]] = -Db[~up]
    G = van_leer(fwd, bwd)
    G[:, mesh.dim:, :] = 0.0
    return G


def material_diag(eps, mu, ncomp=6):
    """Diagonal of M = diag(eps I, mu I) per cell, [ncell, 6]; with the cleaning potentials
    (ncomp = 8) M = diag(eps I, mu I, 1, 1)."""
    mu = np.ones_like(eps) if mu is None else mu
    cols = [eps, eps, eps, mu, mu, mu] + [np.ones_like(eps)] * (ncomp - 6)
    return np.stack(cols, axis=1)


def face_fluxes(mesh: FVMesh, V, m, C, dt, c=1.0, faces=None, phm=None, limiter=None):
    """Global-frame flux F_s . n_s on every face (or on the subset ``faces``), [nf, ncomp].
    limiter = "vanleer" takes the limited Cartesian gradient instead of Green-Gauss."""
    if limiter is None:
        G = green_gauss(mesh, V)
    elif limiter == "vanleer":
        G = limited_gradient(mesh, V)
    else:
        raise ValueError(f"unknown limiter {limiter!r}")
    sel = np.arange(mesh.nface) if faces is None else np.asarray(faces)
    L, R = mesh.L[sel], mesh.R[sel]
    ghost = mesh.boundary[sel]
    Rc = np.maximum(R, 0)
    # piecewise-linear reconstruction at the face centre
    Vl = V[L] + np.einsum("fj,fjc->fc", mesh.dL[sel], G[L])
    Vr = V[Rc] + np.einsum("fj,fjc->fc", mesh.dR[sel], G[Rc])
    Gr, mr = G[Rc], m[Rc]
    pec = mesh.pec_faces()[sel]
    if pec.any():
        # PEC wall: the high side is the mirror ghost of the low side, with its materials
        n = mesh.normal[sel][pec]
        Vr = Vr.copy(); Gr = Gr.copy(); mr = mr.copy()
        Vr[pec] = pec_mirror(n, Vl[pec])
        Gr[pec] = pec_mirror_grad(n, G[L[pec]])
        mr[pec] = m[L[pec]]
    T = rotation(mesh.normal[sel])
    Fl = face_flux_local(_rot_vec6(T, Vl), _rot_grad(T, G[L]), m[L],
                         _rot_vec6(T, Vr), _rot_grad(T, Gr), mr, ghost, C, dt, c, mesh.dim, phm)
    return _rot_vec6_back(T, Fl)


def step(mesh: FVMesh, V, m, dt, C, c=1.0, jz=None, phm=None, limiter=None):
    """One GKS step: U^{n+1} = U^n - dt/|Omega_i| sum_s +-|l_s| F_s + dt S_i, S = (-J, 0).

    V [ncell, 6] primitive state at t^n ([ncell, 8] with phi, psi for the cleaning system,
    phm = (chi, gamma)); m the matching material diagonal; jz [ncell] current density J_z at
    t^n (or None).  Returns V^{n+1}."""
    F = face_fluxes(mesh, V, m, C, dt, c, phm=phm, limiter=limiter)
    flux = F * mesh.area[:, None]
    inter = mesh.R >= 0
    net = _scatter_add(mesh.ncell, mesh.L, flux)
    net -= _scatter_add(mesh.ncell, mesh.R[inter], flux[inter])
    U = m * V
    U_new = U - (dt / mesh.vol)[:, None] * net
    if jz is not None:
        U_new[:, 2] = U_new[:, 2] - dt * jz
    return U_new / m


# --------------------------------------------------------------------------------------------
# Diagnostics: energy and the probe objective (not in the paper; plain definitions)
# --------------------------------------------------------------------------------------------

def energy(mesh: FVMesh, V, m):
    """Electromagnetic energy 1/2 sum_i |Omega_i| (eps |E|^2 + mu |H|^2) (plus phi^2 + psi^2
    for the cleaning system, the quadratic form its equations conserve)."""
    return 0.5 * float(np.sum(mesh.vol[:, None] * m * V * V))


def probe_term(mesh: FVMesh, V, probe, dt):
    """dt * sum_{i in probe} |Omega_i| Ez_i^2 (one step's contribution to J)."""
    return dt * np.sum(mesh.vol[probe] * V[probe, 2] * V[probe, 2])


# --------------------------------------------------------------------------------------------
# Convenience drivers
# --------------------------------------------------------------------------------------------

TM_COMPONENTS = (2, 3, 4)     # (Ez, Hx, Hy) inside (Ex, Ey, Ez, Hx, Hy, Hz)
TM_PSI_COMPONENTS = (2, 3, 4, 7)   # (Ez, Hx, Hy, psi) inside (E, H, phi, psi)


def fields_to_state(fields, dim):
    """[ncomp][ncell] user fields -> oracle state.  2-D: (Ez, Hx, Hy) -> [ncell, 6] with TM in
    the (E, H) slots, or (Ez, Hx, Hy, psi) -> [ncell, 8]; 3-D: 6 or 8 rows (E, H[, phi, psi])."""
    fields = np.asarray(fields)
    if dim == 3:
        return np.ascontiguousarray(fields.T)
    width = 8 if fields.shape[0] == 4 else 6
    comps = TM_PSI_COMPONENTS if width == 8 else TM_COMPONENTS
    V = np.zeros((fields.shape[1], width), dtype=fields.dtype)
    V[:, list(comps)] = fields.T
    return V


def state_to_fields(V, dim):
    if dim == 3:
        return np.ascontiguousarray(V.T)
    comps = TM_PSI_COMPONENTS if V.shape[1] == 8 else TM_COMPONENTS
    return np.ascontiguousarray(V[:, list(comps)].T)


def source_signal(t, A, f0, t0, s):
    """Gaussian-modulated sinusoid of the line-source workloads."""
    return A * math.exp(-(((t - t0) / s) ** 2)) * math.sin(2.0 * math.pi * f0 * (t - t0))


def source_signal_cw(t, A, f0, t0):
    """Time-harmonic current of the oscillating dipole (Sec. 5.4): A cos(2 pi f0 (t - t0)),
    switched on at t0."""
    return A * math.cos(2.0 * math.pi * f0 * (t - t0)) if t >= t0 else 0.0


def run(mesh: FVMesh, fields, eps, mu, cfl, nsteps, kappa=0.0, c=1.0, jz_mask=None,
        src=None, t0=0.0, dt=None, probe=None, callback=None, waveform="gauss_sine", phm=None,
        limiter=None):
    """Advance ``nsteps`` steps from user fields [ncomp][ncell].  Returns (fields, info) with
    info = {dt, t, J} (J only when ``probe`` is given: sum over n = 1..N of the probe term).
    The source is jz_mask times source_signal(t, *src) ("gauss_sine") or
    source_signal_cw(t, *src) ("cw").  phm = (chi, gamma) runs the divergence-cleaning system of
    Sec. 2.1 (fields then carry psi in 2-D, phi and psi in 3-D).  limiter = "vanleer" limits
    the slopes (limited_gradient)."""
    signal = source_signal_cw if waveform == "cw" else source_signal
    dim = mesh.dim
    V = fields_to_state(fields, dim)
    m = material_diag(np.asarray(eps), None if mu is None else np.asarray(mu), V.shape[1])
    if dt is None:
        dt = time_step(mesh, cfl, c)
    C = time_coefficients(dt, kappa * dt)
    J = 0.0
    for n in range(nsteps):
        t = t0 + n * dt
        jz = None
        if jz_mask is not None:
            jz = jz_mask * signal(t, *src)
        V = step(mesh, V, m, dt, C, c, jz, phm, limiter)
        if probe is not None:
            J = J + probe_term(mesh, V, probe, dt)
        if callback is not None:
            callback(n + 1, V)
    return state_to_fields(V, dim), {"dt": dt, "t": t0 + nsteps * dt, "J": J}
