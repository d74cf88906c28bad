"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU needed).

Each test names the passage it checks.  None of them re-types the oracle's own formula: the
checks use independent derivations (closed forms written with cross products), exact rational
arithmetic, high-precision quadrature, printed values from the paper, or invariants."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import gks_oracle as go
from paper_2412_16845_gb300 import workloads as wl
from tests import closed_form as cf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_state(rng, n):
    return rng.standard_normal((n, 6))


# ---------------------------------------------------------------------------- Sec. 2.1 / 2.2

@pytest.mark.parametrize("dim", [2, 3])
def test_equilibrium_compatibility(dim):
    """Sec. 2.2: sum_k g_k = U and sum_k u_k^j g_k = F_j(U) for the D3Q4 / D2Q4 lattice."""
    rng = np.random.default_rng(1)
    V = _rand_state(rng, 50)
    m = np.abs(rng.standard_normal((50, 6))) + 0.5
    for c in (1.0, 1.7):
        u = go.lattice(dim, c)
        g = [go.equilibrium(m * V, V, u[k], c) for k in range(4)]
        assert np.allclose(sum(g), m * V, atol=1e-14, rtol=0)
        for j in range(dim):
            assert np.allclose(sum(u[k, j] * g[k] for k in range(4)), go.flux_dir(j, V),
                               atol=1e-14, rtol=0)
        gg = go.equilibria(m * V, V, u, c)
        for k in range(4):
            assert np.array_equal(gg[k], g[k])


def test_lattice_is_d3q4():
    """Sec. 2.2: four velocities c(+-1,+-1,+-1) with sign product +1; the 2-D set is their
    projection (D2Q4)."""
    u = go.lattice(3, 2.0)
    assert u.shape == (4, 3)
    assert np.all(np.abs(u) == 2.0)
    assert np.all(np.prod(np.sign(u), axis=1) == 1.0)
    assert len({tuple(r) for r in u}) == 4
    u2 = go.lattice(2, 1.0)
    assert {tuple(r[:2]) for r in u2} == {(1, 1), (1, -1), (-1, 1), (-1, -1)}


def test_flux_functions_are_maxwell():
    """Sec. 2.1: F_j = A_j U; sum_j d_j F_j must give dE/dt = curl H, dH/dt = -curl E.  Checked
    against Maxwell's flux written with cross products, F_e = (-e x H, e x E)."""
    rng = np.random.default_rng(2)
    V = _rand_state(rng, 20)
    for j in range(3):
        e = [0.0, 0.0, 0.0]
        e[j] = 1.0
        ref = np.array([cf.flux_along(e, list(v)) for v in V])
        assert np.array_equal(go.flux_dir(j, V), ref)
    # a linear field V(x) = V0 + x_j G_j: -sum_j F_j(G_j) = (curl H, -curl E)
    G = rng.standard_normal((3, 6))
    div_F = sum(go.flux_dir(j, G[j]) for j in range(3))
    curl = lambda A: np.array([G[1][A + 2] - G[2][A + 1], G[2][A + 0] - G[0][A + 2],
                               G[0][A + 1] - G[1][A + 0]])
    assert np.allclose(-div_F[:3], curl(3), atol=1e-15)
    assert np.allclose(-div_F[3:], -curl(0), atol=1e-15)


# ---------------------------------------------------------------------------- Sec. 3.1 coefficients

@pytest.mark.parametrize("kappa", [1e-6, 1e-3, 0.05, 0.3, 0.5, 0.51, 1.0, 3.0, 1e3])
def test_coefficients_against_quadrature(kappa):
    """Sec. 3.1: C_i = int_0^dt c_i(t) dt with c1 = 1 - e^{-t/tau}, c2 = (tau + t)e^{-t/tau} -
    tau, c3 = t + tau(e^{-t/tau} - 1), c4 = e^{-t/tau}, c5 = t e^{-t/tau}; evaluated by
    50-digit quadrature of the integrands."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    dt = 0.0137
    tau = kappa * dt
    C = go.time_coefficients(dt, tau)
    T = mp.mpf(tau)
    ints = [lambda t: 1 - mp.e ** (-t / T),
            lambda t: (T + t) * mp.e ** (-t / T) - T,
            lambda t: t + T * (mp.e ** (-t / T) - 1),
            lambda t: mp.e ** (-t / T),
            lambda t: t * mp.e ** (-t / T)]
    for Ci, f in zip(C, ints):
        ref = mp.quad(f, [0, mp.mpf(dt)])
        assert abs(Ci - float(ref)) <= 2e-15 * max(abs(float(ref)), 1e-300) + 1e-30


def test_coefficient_identities_and_limits():
    """C1 + C4 = dt and C3 - C2 + C5 = dt^2/2 (from the printed closed forms); tau -> 0 gives
    (dt, 0, dt^2/2, 0, 0) (Sec. 4.1 non-viscous limit); small tau gives the leading terms dt,
    -tau dt, dt^2/2 - tau dt (Sec. 4.1 viscous limit)."""
    dt = 0.01
    for kappa in (1e-8, 1e-3, 1.0, 1e3):
        C = go.time_coefficients(dt, kappa * dt)
        assert abs(C[0] + C[3] - dt) <= 1e-17
        assert abs(C[2] - C[1] + C[4] - 0.5 * dt * dt) <= 1e-19
    assert go.time_coefficients(dt, 0.0) == (dt, 0.0, 0.5 * dt * dt, 0.0, 0.0)
    tau = 1e-4 * dt
    C = go.time_coefficients(dt, tau)
    assert abs(C[0] - dt) < 2 * tau
    assert abs(C[1] + tau * dt) < 3 * tau * tau
    assert abs(C[2] - (0.5 * dt * dt - tau * dt)) < 2 * tau * tau


# ---------------------------------------------------------------------------- Sec. 3.1 rotation

def test_rotation_properties():
    """Sec. 3.1: T' is a rotation (orthonormal, det +1) whose first row is n; T'(e_x) = I;
    n_1 = -1 gives diag(-1, -1, 1)."""
    rng = np.random.default_rng(3)
    n = rng.standard_normal((200, 3))
    n[:5] = [[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, 0, -1], [-1 + 1e-9, 1e-4, 0]]
    n /= np.linalg.norm(n, axis=1)[:, None]
    T = go.rotation(n)
    eye = np.einsum("fab,fcb->fac", T, T)
    assert np.allclose(eye, np.eye(3), atol=1e-12)
    assert np.allclose(np.linalg.det(T), 1.0, atol=1e-12)
    assert np.allclose(T[:, 0, :], n, atol=0)
    assert np.array_equal(T[0], np.eye(3))
    assert np.array_equal(T[1], np.diag([-1.0, -1.0, 1.0]))


# ---------------------------------------------------------------------------- flux: literal vs closed form

@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("ghost", [False, True])
@pytest.mark.parametrize("kappa", [0.0, 0.05, 1.0, 1e3])
def test_literal_flux_matches_closed_form(dim, ghost, kappa):
    """The oracle's per-velocity flux (Sec. 3.1) equals the independently derived closed form
    (tests/closed_form.py) for random states, gradients, materials and normals."""
    rng = np.random.default_rng(10 + dim + 2 * ghost)
    nf = 40
    if dim == 2:
        a = rng.uniform(0, 2 * np.pi, nf)
        nrm = np.stack([np.cos(a), np.sin(a), np.zeros(nf)], axis=1)
        nrm[:4] = [[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0]]
    else:
        nrm = rng.standard_normal((nf, 3))
        nrm[:6] = [[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]]
        nrm /= np.linalg.norm(nrm, axis=1)[:, None]
    Vl, Vr = _rand_state(rng, nf), _rand_state(rng, nf)
    Gl, Gr = rng.standard_normal((nf, 3, 6)), rng.standard_normal((nf, 3, 6))
    if dim == 2:
        Gl[:, 2] = 0.0
        Gr[:, 2] = 0.0
    ml = np.repeat(rng.uniform(1, 4, (nf, 2)), 3, axis=1)
    mr = np.repeat(rng.uniform(1, 4, (nf, 2)), 3, axis=1)
    dt, c = 0.013, 1.3
    C = go.time_coefficients(dt, kappa * dt)
    g = np.full(nf, ghost)
    T = go.rotation(nrm)
    lit = go._rot_vec6_back(T, go.face_flux_local(
        go._rot_vec6(T, Vl), go._rot_grad(T, Gl), ml,
        go._rot_vec6(T, Vr), go._rot_grad(T, Gr), mr, g, C, dt, c, dim))
    for f in range(nf):
        frame = [list(T[f, 0]), list(T[f, 1]), list(T[f, 2])]
        ref = cf.face_flux(frame, list(Vl[f]), [list(r) for r in Gl[f]], list(ml[f]),
                           list(Vr[f]), [list(r) for r in Gr[f]], list(mr[f]), ghost, C, dt, c,
                           dim)
        assert np.allclose(lit[f], ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_flux_frame_independent_at_kappa_zero():
    """At tau = 0 only <u g0> and <u g_t> remain; both are rotation-covariant, so any face
    frame with the same normal gives the same flux (used by the exact brute-force test)."""
    rng = np.random.default_rng(5)
    n = np.array([0.0, 1.0, 0.0])
    Vl, Vr = list(rng.standard_normal(6)), list(rng.standard_normal(6))
    Gl = [list(r) for r in rng.standard_normal((3, 6))]
    Gr = [list(r) for r in rng.standard_normal((3, 6))]
    m = [2.0] * 3 + [1.0] * 3
    C = go.time_coefficients(0.01, 0.0)
    f1 = cf.face_flux((list(n), [-1, 0, 0], [0, 0, 1]), Vl, Gl, m, Vr, Gr, m, False, C, 0.01,
                      1.0, 3)
    f2 = cf.face_flux((list(n), [0, 0, 1], [1, 0, 0]), Vl, Gl, m, Vr, Gr, m, False, C, 0.01,
                      1.0, 3)
    assert np.allclose(f1, f2, atol=1e-14)


def _tem_1d_flux(Vl, Vr, kappa, c, eps, mu, ghost=False):
    """Oracle flux through an x-face for x-only data with zero gradients."""
    Z = np.zeros((1, 3, 6))
    m = np.array([[eps] * 3 + [mu] * 3])
    C = go.time_coefficients(0.01, kappa * 0.01)
    return go.face_flux_local(np.array([Vl]), Z, m, np.array([Vr]), Z, m, np.array([ghost]), C,
                              0.01, c, 3)[0]


def test_collisionless_limit_equals_fvs():
    """Sec. 4.1: for the 1-D TEM mode the kinetic split fluxes equal A+ U and A- U with the
    printed matrices, so the GKS flux of piecewise-constant data is the FVS upwind flux
    (1/2)A(U_L + U_R) - (1/2)|A|(U_R - U_L) (Sec. 3.3) for every tau, and the non-reflecting
    flux is A+ U_L (Sec. 3.3, last paragraph)."""
    rows = np.loadtxt(os.path.join(GOLDEN, "paper_sec41_d1q2_split.txt"))
    rng = np.random.default_rng(7)
    for row in rows:
        c = row[0]
        Ap = row[1:5].reshape(2, 2)
        Am = row[5:9].reshape(2, 2)
        A = Ap + Am
        absA = Ap - Am
        # c^2 = 1/(eps0 mu0): take eps0 = mu0 = 1/c; paper state (E_y, B_z), ours (eps E_y, mu H_z)
        eps = mu = 1.0 / c
        for _ in range(5):
            pl, pr = rng.standard_normal(2), rng.standard_normal(2)   # (E_y, B_z) left / right
            Vl = np.zeros(6); Vl[1] = pl[0]; Vl[5] = pl[1] / mu
            Vr = np.zeros(6); Vr[1] = pr[0]; Vr[5] = pr[1] / mu
            fvs = 0.5 * A @ (pl + pr) - 0.5 * absA @ (pr - pl)
            for kappa in (0.0, 0.05, 1.0, 1e3):
                F = _tem_1d_flux(Vl, Vr, kappa, c, eps, mu)
                # our D_y flux is eps0 times the paper's E_y flux; the B_z flux is the same
                assert np.allclose([F[1] / eps, F[5]], fvs, rtol=1e-12, atol=1e-14)
                Fb = _tem_1d_flux(Vl, Vr, kappa, c, eps, mu, ghost=True)
                assert np.allclose([Fb[1] / eps, Fb[5]], Ap @ pl, rtol=1e-12, atol=1e-14)


def test_1d_flux_independent_of_tau():
    """For x-only data with |u_n| = c the free-transport and equilibrium parts coincide, so the
    GKS flux does not depend on tau (follows from C1 + C4 = dt and C3 - C2 + C5 = dt^2/2)."""
    rng = np.random.default_rng(8)
    Vl, Vr = np.zeros((1, 6)), np.zeros((1, 6))
    Vl[0, [1, 5]] = rng.standard_normal(2)
    Vr[0, [1, 5]] = rng.standard_normal(2)
    Gl, Gr = np.zeros((1, 3, 6)), np.zeros((1, 3, 6))
    Gl[0, 0, [1, 5]] = rng.standard_normal(2)
    Gr[0, 0, [1, 5]] = rng.standard_normal(2)
    m = np.ones((1, 6))
    F = [go.face_flux_local(Vl, Gl, m, Vr, Gr, m, np.array([False]),
                            go.time_coefficients(0.01, k * 0.01), 0.01, 1.0, 3)
         for k in (0.0, 0.05, 1.0, 1e3)]
    for f in F[1:]:
        assert np.allclose(f, F[0], rtol=1e-10, atol=1e-13)


# ---------------------------------------------------------------------------- brute force, exact

def test_exact_rational_step_3x3():
    """A whole 2-D TM step on a 3x3 periodic grid with rational fields and materials at tau = 0,
    computed in exact rational arithmetic (central differences = Green-Gauss on a uniform grid,
    the closed-form flux, the FV update of Sec. 3.1), against the oracle's FP64 step."""
    rng = np.random.default_rng(11)
    n = 3
    h = Fraction(1, 3)
    dt = Fraction(1, 7)
    num = rng.integers(-9, 10, size=(n * n, 3))
    den = rng.integers(1, 6, size=(n * n, 3))
    ez = [Fraction(int(a), int(b)) for a, b in zip(num[:, 0], den[:, 0])]
    hx = [Fraction(int(a), int(b)) for a, b in zip(num[:, 1], den[:, 1])]
    hy = [Fraction(int(a), int(b)) for a, b in zip(num[:, 2], den[:, 2])]
    eps = [Fraction(int(v), 2) for v in rng.integers(2, 9, size=n * n)]
    Z = Fraction(0)
    V = [[Z, Z, ez[i], hx[i], hy[i], Z] for i in range(n * n)]
    m = [[eps[i]] * 3 + [Fraction(1)] * 3 for i in range(n * n)]
    idx = lambda i, j: (i % n) + n * (j % n)
    G = []
    for j in range(n):
        for i in range(n):
            gx = [(a - b) / (2 * h) for a, b in zip(V[idx(i + 1, j)], V[idx(i - 1, j)])]
            gy = [(a - b) / (2 * h) for a, b in zip(V[idx(i, j + 1)], V[idx(i, j - 1)])]
            G.append([gx, gy, [Z] * 6])
    C = (dt, Z, dt * dt / 2, Z, Z)
    frames = {0: ([1, 0, 0], [0, 1, 0], [0, 0, 1]), 1: ([0, 1, 0], [-1, 0, 0], [0, 0, 1])}
    net = [[Z] * 6 for _ in range(n * n)]
    for j in range(n):
        for i in range(n):
            for ax in (0, 1):
                L = idx(i, j)
                R = idx(i + 1, j) if ax == 0 else idx(i, j + 1)
                e = frames[ax][0]
                Vl = [v + h / 2 * d for v, d in zip(V[L], cf.dir_deriv(G[L], e))]
                Vr = [v - h / 2 * d for v, d in zip(V[R], cf.dir_deriv(G[R], e))]
                F = cf.face_flux(frames[ax], Vl, G[L], m[L], Vr, G[R], m[R], False, C, dt,
                                 Fraction(1), 2)
                net[L] = [a + h * f for a, f in zip(net[L], F)]
                net[R] = [a - h * f for a, f in zip(net[R], F)]
    Vnew = [[(m[i][c] * V[i][c] - dt / (h * h) * net[i][c]) / m[i][c] for c in range(6)]
            for i in range(n * n)]
    mesh = go.cartesian_mesh((n, n), (0.0, 0.0), (1.0, 1.0), ("periodic",) * 4)
    Vf = np.array([[float(x) for x in v] for v in V])
    mf = np.array([[float(x) for x in r] for r in m])
    out = go.step(mesh, Vf, mf, float(dt), tuple(float(x) for x in C))
    ref = np.array([[float(x) for x in v] for v in Vnew])
    assert np.allclose(out, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


# ---------------------------------------------------------------------------- whole scheme

def _plane_wave_error(n, T=1.5625):
    w = wl.config1_periodic_tm(n, with_pulse=False)
    mesh = go.cartesian_mesh(w.n, w.lo, w.hi, w.bc)
    dt = go.time_step(mesh, 0.5)
    nst = int(round(T / dt))
    f, info = go.run(mesh, w.fields0, w.eps, None, 0.5, nst)
    x, y = wl.cell_centres_2d(n, n)
    ex = wl.plane_wave_tm(x, y, info["t"])
    return np.sqrt(np.mean((f - ex) ** 2))


@pytest.mark.slow
def test_plane_wave_second_order():
    """Exact oblique TM plane wave (Sec. 5.1 solution, rotated): L2 error falls at order
    2 +- 0.1 under refinement 32 -> 64 -> 128 at CFL 0.5, T = 1.5625."""
    e = [_plane_wave_error(n) for n in (32, 64, 128)]
    orders = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert all(abs(o - 2.0) <= 0.1 for o in orders), (e, orders)
    assert e[-1] < 3e-3


def test_plane_wave_order_coarse():
    """Fast version of the order check (32 -> 64)."""
    e = [_plane_wave_error(n) for n in (32, 64)]
    assert abs(math.log2(e[0] / e[1]) - 2.0) <= 0.15, e


def test_cavity_mode_within_factor_of_table3():
    """Sec. 5.2, Table 3: the TM mode E_z = sin(8 pi x) sin(8 pi y) cos(8 sqrt2 pi t) at
    t = 1.775, CFL 0.5, 50 x 50.  The mode is also an exact solution on the periodic unit
    square; there the oracle's errors land within a factor 1.3 of the printed ones (the paper's
    wall treatment for Cartesian GKS is not specified, so closer agreement is not expected)."""
    tab = np.loadtxt(os.path.join(GOLDEN, "paper_table3_tm_cavity.txt"))
    a, w0 = 8 * np.pi, 8 * math.sqrt(2) * np.pi
    N = 50
    mesh = go.cartesian_mesh((N, N), (0, 0), (1, 1), ("periodic",) * 4)
    x, y = mesh.centroid[:, 0], mesh.centroid[:, 1]
    f = np.zeros((3, mesh.ncell))
    f[0] = np.sin(a * x) * np.sin(a * y)
    nst = int(math.ceil(1.775 / (0.5 / N) - 1e-9))
    out, info = go.run(mesh, f, np.ones(mesh.ncell), None, 0.5, nst, dt=1.775 / nst)
    e = out[0] - np.sin(a * x) * np.sin(a * y) * math.cos(w0 * info["t"])
    # The printed L-inf/L1 ratio (1.59 ~ pi/2) is that of a 1-D sine, i.e. the paper's norms
    # look line-based; only the L1 value is compared.
    l1 = np.abs(e).mean()
    assert tab[0, 1] / 1.3 <= l1 <= tab[0, 1] * 1.3, (l1, tab[0])


@pytest.mark.parametrize("cfl", [0.5, 0.4])
@pytest.mark.parametrize("kappa", [0.0, 0.05, 1.0])
def test_grid_aligned_3d_update_is_fromm(cfl, kappa):
    """Sec. 5.1 setting (3-D grid, wave along x): for the right-moving TEM mode E_z = w,
    H_y = -w the 3-D step is Fromm's scheme at Courant number nu, exactly:
    w_j <- w_j - nu (w_j - w_{j-1}) - nu (1 - nu)/4 (w_{j+1} - w_j - w_{j-1} + w_{j-2}),
    whatever kappa (the 1-D flux does not depend on tau), with the other components staying 0.
    A dropped or mis-signed term of the 3-D face flux or of the Green-Gauss gradient along the
    normal breaks the equality."""
    N = 12
    rng = np.random.default_rng(3)
    mesh = go.cartesian_mesh((N, 1, 1), (0, 0, 0), (1, 1 / N, 1 / N), ("periodic",) * 6)
    w = rng.standard_normal(N)
    V = np.zeros((N, 6))
    V[:, 2], V[:, 4] = w, -w
    dt = cfl / N
    Vn = go.step(mesh, V, go.material_diag(np.ones(N), None), dt,
                 go.time_coefficients(dt, kappa * dt))
    nu = cfl
    wm1, wm2, wp1 = np.roll(w, 1), np.roll(w, 2), np.roll(w, -1)
    fromm = w - nu * (w - wm1) - nu * (1 - nu) / 4 * (wp1 - w - wm1 + wm2)
    assert np.abs(Vn[:, 2] - fromm).max() <= 1e-14
    assert np.abs(Vn[:, 4] + fromm).max() <= 1e-14
    assert np.abs(Vn[:, [0, 1, 3, 5]]).max() == 0.0


def test_table1_grid_aligned_wave_is_third_order():
    """Sec. 5.1, Table 1 (golden file): E_z = cos 2 pi (x - t), B_y = -E_z on the periodic unit
    cube, CFL 0.5, t = 1, N = 20 .. 160.  The oracle's errors are not the printed ones: for this
    wave the scheme is Fromm's (test above), third order at Courant number 1/2, so its L1, L2
    and L-inf errors fall at order 3 +- 0.05 and sit below the table's second-order errors by a
    factor that starts near 4 at N = 20 and doubles with every refinement (to within the
    table's own order, 1.92 .. 2.02).  No reading of the CFL reproduces the table; this pins
    the measured relation instead."""
    tab = np.loadtxt(os.path.join(GOLDEN, "paper_table1_plane_wave.txt"))
    errs = []
    for N in tab[:, 0].astype(int):
        mesh = go.cartesian_mesh((N, 1, 1), (0, 0, 0), (1, 1 / N, 1 / N), ("periodic",) * 6)
        x = mesh.centroid[:, 0]
        f = np.zeros((6, N))
        f[2] = np.cos(2 * np.pi * x)
        f[4] = -f[2]
        out, info = go.run(mesh, f, np.ones(N), None, 0.5, 2 * N, dt=0.5 / N)
        assert abs(info["t"] - 1.0) < 1e-12
        e = out[2] - np.cos(2 * np.pi * (x - info["t"]))
        errs.append((np.abs(e).mean(), np.sqrt((e * e).mean()), np.abs(e).max()))
    errs = np.array(errs)
    orders = np.log2(errs[:-1] / errs[1:])
    assert np.all(np.abs(orders - 3.0) <= 0.05), orders
    ratio = tab[:, 1:4] / errs
    assert np.all((ratio[0] > 3.5) & (ratio[0] < 5.0)), ratio[0]
    assert np.all(np.abs(ratio[1:] / ratio[:-1] - 2.0) <= 0.15), ratio


def _oblique_symbol(N, cfl, kappa=0.0):
    """The oracle's one-step amplification matrix G for the Fourier mode exp(2 pi i (x + y + z))
    on the periodic N^3 unit cube (the step applied to the six single-component modes; the step
    is linear and translation invariant, which the check inside confirms cell by cell)."""
    mesh = go.cartesian_mesh((N, N, N), (0, 0, 0), (1, 1, 1), ("periodic",) * 6)
    ph = np.exp(2j * np.pi * mesh.centroid.sum(axis=1))
    dt = go.time_step(mesh, cfl)
    C = go.time_coefficients(dt, kappa * dt)
    m = go.material_diag(np.ones(mesh.ncell), None).astype(complex)
    G = np.zeros((6, 6), complex)
    for c in range(6):
        V = np.zeros((mesh.ncell, 6), complex)
        V[:, c] = ph
        Vn = go.step(mesh, V, m, dt, C) / ph[:, None]
        assert np.abs(Vn - Vn[0]).max() <= 1e-12
        G[:, c] = Vn[0]
    return G, dt


def test_oblique_3d_plane_wave_second_order():
    """Sec. 5.1 in three dimensions: the exact oblique plane wave E = a e^{i(k.x - |k| t)},
    H = (k/|k|) x E with k = 2 pi (1, 1, 1) on the periodic unit cube, CFL 0.4 (the 3-D
    workload's), t = 0.5.  The oracle's solution G^n u0 (n = t/dt steps of the mode) converges
    at order 2 +- 0.1 from 16^3 to 32^3."""
    k = 2 * np.pi * np.ones(3)
    khat = k / np.linalg.norm(k)
    a = np.array([1.0, -1.0, 0.0]) / math.sqrt(2.0)
    u0 = np.concatenate([a, np.cross(khat, a)]).astype(complex)
    T = 0.5
    err = []
    for N in (16, 32):
        G, dt = _oblique_symbol(N, 0.4)
        n = int(round(T / dt))
        assert abs(n * dt - T) < 1e-12
        exact = np.exp(-1j * np.linalg.norm(k) * T) * u0
        err.append(np.linalg.norm(np.linalg.matrix_power(G, n) @ u0 - exact))
    order = math.log2(err[0] / err[1])
    assert abs(order - 2.0) <= 0.1, (err, order)
    assert err[1] < 0.03


def _smooth_random_fields(rng, mesh, ncomp_modes=3):
    x = mesh.centroid
    V = np.zeros((mesh.ncell, 6))
    for c in range(6):
        for _ in range(ncomp_modes):
            k = rng.integers(-2, 3, size=3) * 2 * np.pi
            V[:, c] += rng.standard_normal() * np.cos(x @ k + rng.uniform(0, 6.3))
    if mesh.dim == 2:
        V[:, [0, 1, 5]] = 0.0
    return V


@pytest.mark.parametrize("dim,cfl", [(2, 0.5), (3, 0.4)])
@pytest.mark.parametrize("kappa", [0.0, 0.05])
def test_energy_bounded_and_conservation_periodic(dim, cfl, kappa):
    """Periodic grids with variable eps: sum |Omega| U is conserved to round-off (the FV update
    telescopes over periodic faces) and the energy stays bounded.  The energy is *not* monotone
    step by step: the amplification matrices are non-normal (see the next test), so transient
    growth of up to sigma_max per step is possible."""
    rng = np.random.default_rng(20 + dim)
    n = (12, 10) if dim == 2 else (8, 6, 5)
    mesh = go.cartesian_mesh(n, (0.0,) * dim, (1.0,) * dim, ("periodic",) * (2 * dim))
    V = _smooth_random_fields(rng, mesh)
    eps = rng.uniform(1.0, 3.0, mesh.ncell)
    m = go.material_diag(eps, None)
    dt = go.time_step(mesh, cfl)
    C = go.time_coefficients(dt, kappa * dt)
    E0 = go.energy(mesh, V, m)
    tot0 = (mesh.vol[:, None] * m * V).sum(axis=0)
    for _ in range(30):
        V = go.step(mesh, V, m, dt, C)
        assert go.energy(mesh, V, m) <= 1.2 * E0
    tot = (mesh.vol[:, None] * m * V).sum(axis=0)
    assert np.allclose(tot, tot0, atol=1e-13)


def _amplification(dim, n, cfl, kappa):
    shape = (n,) * dim
    mesh = go.cartesian_mesh(shape, (0.0,) * dim, (1.0,) * dim, ("periodic",) * (2 * dim))
    m = np.ones((mesh.ncell, 6))
    dt = go.time_step(mesh, cfl)
    C = go.time_coefficients(dt, kappa * dt)
    comps = [2, 3, 4] if dim == 2 else list(range(6))
    modes = np.array(np.meshgrid(*[np.arange(n)] * dim, indexing="ij")).reshape(dim, -1).T
    out_G = []
    for kk in modes:
        k = np.zeros(3)
        k[:dim] = 2 * np.pi * kk
        phase = np.exp(1j * (mesh.centroid @ k))
        Gk = np.zeros((len(comps), len(comps)), dtype=complex)
        for a, ca in enumerate(comps):
            V = np.zeros((mesh.ncell, 6), dtype=complex)
            V[:, ca] = phase
            out = go.step(mesh, V, m, dt, C)
            Gk[:, a] = (out[:, comps] / phase[:, None]).mean(axis=0)
            # the image of a Fourier mode is the same mode (translation invariance)
            assert np.allclose(out[:, comps], np.outer(phase, Gk[:, a]), atol=1e-12)
        out_G.append((kk, Gk))
    return out_G


@pytest.mark.parametrize("dim,n,cfl", [(2, 8, 0.5), (3, 6, 0.4)])
def test_amplification_matrix_spectrum(dim, n, cfl):
    """On a periodic vacuum grid the step is a convolution; applying it to single Fourier modes
    gives the amplification matrix G(k) (3x3 in 2-D TM, 6x6 in 3-D).  At tau = 0 and the
    workloads' CFL every eigenvalue lies in the closed unit disc (von Neumann stable) and k = 0
    is exact; sigma_max(G) exceeds 1 (about 1.14 in 2-D at CFL 0.5, 1.05 in 3-D at CFL 0.4), so
    the discrete energy is bounded but not monotone."""
    rho, smax = 0.0, 0.0
    for kk, Gk in _amplification(dim, n, cfl, 0.0):
        rho = max(rho, np.abs(np.linalg.eigvals(Gk)).max())
        smax = max(smax, np.linalg.svd(Gk, compute_uv=False).max())
        if not kk.any():
            assert np.allclose(Gk, np.eye(Gk.shape[0]), atol=1e-14)
    assert rho <= 1.0 + 1e-12, rho
    assert 1.0 < smax < 1.2, smax


def test_3d_positive_tau_is_unstable_at_cfl_04():
    """With tau > 0 the D3Q4 third moment adds the anisotropic term c(F_w(d_t V) + F_t(d_w V));
    at kappa = tau/dt = 0.05 and CFL 0.4 it pushes some 3-D modes outside the unit disc.  This
    is why kappa = 0 is the default."""
    rho = max(np.abs(np.linalg.eigvals(Gk)).max() for _, Gk in _amplification(3, 6, 0.4, 0.05))
    assert rho > 1.0 + 1e-4, rho


def test_grid_aligned_wave_keeps_divergence_zero():
    """A grid-aligned TM wave (k along x) keeps H_x identically zero, so the discrete divergence
    of H stays exactly zero; and the x-only data never creates y-dependence."""
    n = 16
    mesh = go.cartesian_mesh((n, n), (0, 0), (1, 1), ("periodic",) * 4)
    x, y = mesh.centroid[:, 0], mesh.centroid[:, 1]
    f = wl.plane_wave_tm(x, y, 0.0, kvec=(1.0, 0.0))
    out, _ = go.run(mesh, f, np.ones(mesh.ncell), None, 0.5, 20)
    assert np.all(out[1] == 0.0)
    grid = out[0].reshape(n, n)
    assert np.allclose(grid, grid[0:1, :], atol=1e-15)


def test_discrete_divergence_is_truncation_not_round_off():
    """The update of Sec. 3.1 does not keep the central-difference divergence of H.  H starts as
    the discrete curl of a smooth stream function (div_h H = 0 to round-off); after the same time
    on 32^2 and 64^2 periodic grids (CFL 0.5) div_h H is far above round-off, and it falls by
    about 4x per halving of h: a second-order truncation error the scheme creates, not a growing
    one."""
    def rel_div(n, steps):
        h = 1.0 / n
        mesh = go.cartesian_mesh((n, n), (0, 0), (1, 1), ("periodic",) * 4)
        x, y = mesh.centroid[:, 0], mesh.centroid[:, 1]

        def dx(a):
            return (np.roll(a, -1, axis=1) - np.roll(a, 1, axis=1)) / (2 * h)

        def dy(a):
            return (np.roll(a, -1, axis=0) - np.roll(a, 1, axis=0)) / (2 * h)

        def rel(f):
            a, b = f[1].reshape(n, n), f[2].reshape(n, n)
            return np.linalg.norm(dx(a) + dy(b)) / (np.linalg.norm(dx(a)) + np.linalg.norm(dy(b)))

        psi = (np.sin(2 * np.pi * (x + 2 * y)) + 0.5 * np.cos(2 * np.pi * (3 * x - y))).reshape(n, n)
        f = np.stack([np.cos(2 * np.pi * (2 * x - y)), dy(psi).ravel(), -dx(psi).ravel()])
        out, _ = go.run(mesh, f, np.ones(mesh.ncell), None, 0.5, steps)
        return rel(f), rel(out)

    s0, s32 = rel_div(32, 20)
    _, s64 = rel_div(64, 40)
    assert s0 <= 1e-15
    assert s32 > 1e-3 and s64 > 1e-4                 # measured 9.6e-3 and 2.6e-3
    assert 3.0 <= s32 / s64 <= 5.0, s32 / s64        # measured 3.66 (order 1.87)


def test_nonreflecting_boundary_absorbs_1d_pulse():
    """Sec. 3.1 non-reflecting boundary: a right-moving pulse E_z = f(x - t), H_y = -f leaving
    through the kinetic boundary leaves almost nothing behind (no incoming distribution)."""
    n = 200
    mesh = go.cartesian_mesh((n, 2), (0, 0), (1, 2.0 / n), ("nrbc", "nrbc", "periodic",
                                                           "periodic"))
    x = mesh.centroid[:, 0]
    f = np.zeros((3, mesh.ncell))
    f[0] = np.exp(-((x - 0.7) / 0.05) ** 2)
    f[2] = -f[0]
    E0 = 0.5 * np.sum(mesh.vol * (f ** 2).sum(axis=0))
    out, info = go.run(mesh, f, np.ones(mesh.ncell), None, 0.5, int(0.7 / (0.5 / n)))
    E1 = 0.5 * np.sum(mesh.vol * (out ** 2).sum(axis=0))
    assert E1 < 1e-5 * E0, E1 / E0


# ---------------------------------------------------------------------------- tetrahedral meshes

def test_tet_mesh_geometry():
    """Kuhn split of m^3 hexes: volumes sum to 1, every cell is closed (sum_s n_s |l_s| = 0),
    (4 ntet + nbnd)/2 faces with 2 boundary triangles per boundary square."""
    for m, jit in ((3, 0.0), (4, 0.1)):
        vert, tet = wl.kuhn_tet_mesh(m, jit, wl.rng_for(4))
        mesh = go.tet_mesh(vert, tet)
        assert np.all(mesh.vol > 0)
        assert abs(mesh.vol.sum() - 1.0) < 1e-13
        nb = int(mesh.boundary.sum())
        assert nb == 12 * m * m
        assert mesh.nface == (4 * tet.shape[0] + nb) // 2
        s = np.zeros((mesh.ncell, 3))
        na = mesh.normal * mesh.area[:, None]
        np.add.at(s, mesh.L, na)
        inter = mesh.R >= 0
        np.add.at(s, mesh.R[inter], -na[inter])
        assert np.abs(s).max() < 1e-15
        assert np.all(mesh.L[inter] < mesh.R[inter])
        # normals point from L towards R
        assert np.all(np.einsum("ij,ij->i", mesh.normal[inter],
                                mesh.centroid[mesh.R[inter]] - mesh.centroid[mesh.L[inter]]) > 0)
    # the full-size configuration's counts
    m = 64
    assert 6 * m ** 3 == 1572864 and (4 * 6 * m ** 3 + 12 * m * m) // 2 == 3170304


def test_tet_time_step_matches_cube_rule():
    """dt = CFL h_min / c with h_i = 6 |Omega_i| / sum |l_s|, which is 1 for a unit cube; an
    unjittered Kuhn tet of edge h has h_i = h / (1 + sqrt 2)."""
    vert, tet = wl.kuhn_tet_mesh(4, 0.0, None)
    mesh = go.tet_mesh(vert, tet)
    assert abs(go.time_step(mesh, 1.0) - 0.25 / (1 + math.sqrt(2))) < 1e-15
    cube = go.cartesian_mesh((4, 4, 4), (0,) * 3, (1,) * 3, ("nrbc",) * 6)
    assert abs(go.time_step(cube, 1.0) - 0.25) < 1e-16


def test_tet_energy_decays():
    """Jittered tetrahedra with eps jumps and the non-reflecting boundary at CFL 0.4, tau = 0:
    the energy stays bounded and decays as the fields leave (the tet CFL reading is stable)."""
    kappa = 0.0
    w = wl.config4_tets(m=4, steps=0)
    mesh = go.tet_mesh(w.vert, w.tet)
    rng = np.random.default_rng(30)
    V = _smooth_random_fields(rng, mesh)
    m = go.material_diag(w.eps, None)
    dt = go.time_step(mesh, 0.4)
    C = go.time_coefficients(dt, kappa * dt)
    E0 = go.energy(mesh, V, m)
    for _ in range(60):
        V = go.step(mesh, V, m, dt, C)
        assert go.energy(mesh, V, m) <= 1.2 * E0
    assert go.energy(mesh, V, m) < 0.9 * E0


def test_tet_plane_wave_converges():
    """Unjittered tets, grid-aligned wave along x in a non-reflecting box: the interior error
    after a short time falls at least at first order under refinement (8 -> 16 hexes per edge).
    Green-Gauss with arithmetic face averages (Sec. 3.1) is not exact for linear fields on Kuhn
    tets (face centroids are off the line joining cell centroids), so the reconstruction is only
    first-order accurate there; on Cartesian grids the same rule gives second order."""
    errs = []
    for m in (8, 16):
        vert, tet = wl.kuhn_tet_mesh(m, 0.0, None)
        mesh = go.tet_mesh(vert, tet)
        x = mesh.centroid[:, 0]
        f = np.zeros((6, mesh.ncell))
        f[2] = np.sin(2 * np.pi * x)
        f[4] = -f[2]
        T = 0.125
        dt0 = go.time_step(mesh, 0.4)
        nst = int(math.ceil(T / dt0))
        out, info = go.run(mesh, f, np.ones(mesh.ncell), None, 0.4, nst, dt=T / nst)
        inner = np.all(np.abs(mesh.centroid - 0.5) < 0.5 - T - 0.13, axis=1)
        e = out[2][inner] - np.sin(2 * np.pi * (x[inner] - T))
        errs.append(np.sqrt(np.mean(e ** 2)))
    assert errs[1] < errs[0] / 2.0, errs


# ---------------------------------------------------------------------------- diagnostics

@pytest.mark.parametrize("dim", [2, 3])
def test_energy_of_sampled_waves_closed_form(dim):
    """Energy 1/2 sum |Omega| (eps |E|^2 + mu |H|^2) of E = a cos(2 pi x), H = b sin(2 pi x)
    sampled at the cell centres of a uniform periodic grid: the discrete sums of cos^2 and sin^2
    over a period are exactly N/2, so the energy is (eps a^2 + mu b^2)/4 on the unit square/cube.
    Distinct eps, mu, a, b catch a swapped material, component or a dropped factor 1/2."""
    n = 12
    mesh = go.cartesian_mesh((n,) * dim, (0.0,) * dim, (1.0,) * dim, ("periodic",) * (2 * dim))
    x = mesh.centroid[:, 0]
    a, b, e, m = 1.0, 2.0, 2.5, 1.5
    V = np.zeros((mesh.ncell, 6))
    V[:, 2 if dim == 2 else 1] = a * np.cos(2 * np.pi * x)       # Ez (2-D) or Ey (3-D)
    V[:, 4 if dim == 2 else 5] = b * np.sin(2 * np.pi * x)       # Hy (2-D) or Hz (3-D)
    md = go.material_diag(np.full(mesh.ncell, e), np.full(mesh.ncell, m))
    assert abs(go.energy(mesh, V, md) - 0.25 * (e * a * a + m * b * b)) <= 1e-13


def test_probe_objective_against_exact_wave():
    """J = sum_{n=1}^{N} dt sum_{i in P} |Omega_i| Ez_i^n^2 for the grid-aligned TM plane wave
    Ez = cos 2pi(x - t), Hy = -Ez (Sec. 5.1) on a periodic 64 x 4 grid, probe = the columns
    x < 1/8, N = 32 steps at CFL 0.5 (t = 1/4): equal to the same sum over the exact solution
    within the scheme's error.  The probe's term at t = 0 and at t = 1/4 differ by a factor of
    about 4.5, so counting steps 0..N-1 instead of 1..N moves J by about 4%; a dropped dt or
    |Omega| moves it by orders of magnitude."""
    nx, ny, N = 64, 4, 32
    h = 1.0 / nx
    mesh = go.cartesian_mesh((nx, ny), (0.0, 0.0), (1.0, ny * h), ("periodic",) * 4)
    x, y = mesh.centroid[:, 0], mesh.centroid[:, 1]
    f0 = wl.plane_wave_tm(x, y, 0.0, kvec=(1.0, 0.0))
    probe = np.nonzero(x < 0.125)[0]
    _, info = go.run(mesh, f0, np.ones(mesh.ncell), None, 0.5, N, c=1.0, probe=probe)
    dt = info["dt"]
    assert abs(dt - 0.5 * h) < 1e-15
    xs = x[probe]
    exact = sum(dt * h * h * np.sum(np.cos(2 * np.pi * (xs - k * dt)) ** 2) for k in range(1, N + 1))
    shifted = sum(dt * h * h * np.sum(np.cos(2 * np.pi * (xs - k * dt)) ** 2) for k in range(0, N))
    assert abs(exact - shifted) > 0.02 * exact            # the pin can tell the two apart
    assert abs(info["J"] - exact) <= 1e-3 * exact, (info["J"], exact)


# ---------------------------------------------------------------------------- PEC walls

def _mirror_parity_fields(rng, mesh, modes=3, potentials=False):
    """Random smooth fields with the parities of the PEC mirror about every wall of the unit box:
    along axis a a component is odd (sin) if the mirror negates it (tangential E, normal H) and
    even (cos) if it keeps it (normal E, tangential H).  With potentials=True the cleaning
    potentials follow: phi odd about every wall, psi even."""
    x = mesh.centroid
    ncomp = 8 if potentials else 6
    V = np.zeros((mesh.ncell, ncomp))
    for c in range(ncomp):
        for _ in range(modes):
            k = rng.integers(1, 3, size=3)
            f = rng.standard_normal() * np.ones(mesh.ncell)
            for a in range(mesh.dim):
                if c == 6:
                    odd = True
                elif c == 7:
                    odd = False
                else:
                    # E_c is normal to the a-walls iff c == a; H_{c-3} likewise
                    normal = (c % 3) == a
                    odd = (not normal) if c < 3 else normal
                f = f * (np.sin if odd else np.cos)(2 * np.pi * k[a] * x[:, a])
            V[:, c] += f
    if mesh.dim == 2:
        V[:, [0, 1, 5]] = 0.0
        if potentials:
            V[:, 6] = 0.0
    return V


@pytest.mark.parametrize("dim,kappa,limiter", [(2, 0.0, None), (2, 0.05, None), (3, 0.0, None),
                                               (2, 0.0, "vanleer"), (3, 0.0, "vanleer")])
def test_pec_box_equals_periodic_for_mirror_symmetric_fields(dim, kappa, limiter):
    """Sec. 5.5 wall conditions: a field with the PEC mirror parities about every wall of the
    unit box evolves on the periodic box exactly as in the PEC box (the mirror ghost of a wall
    cell is then its periodic neighbour).  Equality to rounding pins every sign of the mirror,
    of its gradient and of the reconstruction, with the limited slopes too.  (In 3-D the D3Q4
    set is not mirror symmetric for kappa > 0, so only kappa = 0 is compared there.)"""
    rng = np.random.default_rng(41 + dim)
    n = (14, 12) if dim == 2 else (8, 6, 6)
    per = go.cartesian_mesh(n, (0.0,) * dim, (1.0,) * dim, ("periodic",) * (2 * dim))
    pec = go.cartesian_mesh(n, (0.0,) * dim, (1.0,) * dim, ("pec",) * (2 * dim))
    V = _mirror_parity_fields(rng, per)
    f0 = go.state_to_fields(V, dim)
    # materials even about every wall, so that the mirror ghost's materials are its own
    eps = 2.0 + 0.5 * np.prod(np.cos(2 * np.pi * per.centroid[:, :dim]), axis=1)
    steps = 12
    a, _ = go.run(per, f0, eps, None, 0.4, steps, kappa=kappa, limiter=limiter)
    b, _ = go.run(pec, f0, eps, None, 0.4, steps, kappa=kappa, limiter=limiter)
    assert np.max(np.abs(a)) > 0.1
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a)), np.max(np.abs(a - b))


@pytest.mark.parametrize("dim,cfl", [(2, 0.4), (3, 0.3)])
def test_pec_box_equals_periodic_with_cleaning_potentials(dim, cfl):
    """The same equivalence for the cleaning system (Sec. 2.1 with chi, gamma > 0): with phi odd
    and psi even about every wall (the parities their equations impose, given normal E even and
    normal B odd), the PEC box evolves as the periodic one, to rounding.  Pins the mirror of
    the potentials and of their gradients."""
    rng = np.random.default_rng(77 + dim)
    n = (14, 12) if dim == 2 else (8, 6, 6)
    per = go.cartesian_mesh(n, (0.0,) * dim, (1.0,) * dim, ("periodic",) * (2 * dim))
    pec = go.cartesian_mesh(n, (0.0,) * dim, (1.0,) * dim, ("pec",) * (2 * dim))
    V = _mirror_parity_fields(rng, per, potentials=True)
    f0 = go.state_to_fields(V, dim)
    eps = 2.0 + 0.5 * np.prod(np.cos(2 * np.pi * per.centroid[:, :dim]), axis=1)
    phm = (0.7, 0.9)
    a, _ = go.run(per, f0, eps, None, cfl, 10, phm=phm)
    b, _ = go.run(pec, f0, eps, None, cfl, 10, phm=phm)
    assert np.max(np.abs(a[-1])) > 0.01 and np.max(np.abs(a[-2])) > 0.01   # potentials carry signal
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a)), np.max(np.abs(a - b))


def test_pec_cavity_mode_table3():
    """Sec. 5.2, Table 3, on the PEC box itself: E_z = sin(8 pi x) sin(8 pi y) at 50 x 50,
    CFL 0.5, t = 1.775; the L1 error lands within a factor 1.3 of the printed value."""
    tab = np.loadtxt(os.path.join(GOLDEN, "paper_table3_tm_cavity.txt"))
    a, w0 = 8 * np.pi, 8 * math.sqrt(2) * np.pi
    N = 50
    mesh = go.cartesian_mesh((N, N), (0, 0), (1, 1), ("pec",) * 4)
    x, y = mesh.centroid[:, 0], mesh.centroid[:, 1]
    f = np.zeros((3, mesh.ncell))
    f[0] = np.sin(a * x) * np.sin(a * y)
    nst = int(math.ceil(1.775 / (0.5 / N) - 1e-9))
    out, info = go.run(mesh, f, np.ones(mesh.ncell), None, 0.5, nst, dt=1.775 / nst)
    e = out[0] - np.sin(a * x) * np.sin(a * y) * math.cos(w0 * info["t"])
    l1 = np.abs(e).mean()
    assert tab[0, 1] / 1.3 <= l1 <= tab[0, 1] * 1.3, (l1, tab[0])


def test_pec_wall_reflects_tem_pulse():
    """A TEM pulse E_z = f(x - t), H_y = -f (Sec. 5.1 convention) hits a PEC wall at x = 1 and
    comes back: at t = 1 the exact field is E_z = H_y = -f(x) (tangential E reflects with
    coefficient -1, the wave now runs along -x).  The energy stays (a non-reflecting wall would
    absorb it)."""
    nx, ny = 200, 2
    h = 1.0 / nx
    res = {}
    for wall in ("pec", "nrbc"):
        mesh = go.cartesian_mesh((nx, ny), (0.0, 0.0), (1.0, ny * h), ("nrbc", wall, "periodic", "periodic"))
        x = mesh.centroid[:, 0]
        f = np.exp(-(((x - 0.5) / 0.05) ** 2))
        f0 = np.zeros((3, mesh.ncell))
        f0[0], f0[2] = f, -f
        out, info = go.run(mesh, f0, np.ones(mesh.ncell), None, 0.5, 400)
        assert abs(info["t"] - 1.0) < 1e-12
        res[wall] = (out, f)
    out, f = res["pec"]
    err = np.sqrt(np.sum((out[0] + f) ** 2 + (out[2] + f) ** 2) / np.sum(2 * f * f))
    assert err <= 0.05, err
    assert np.max(np.abs(out[1])) <= 1e-12
    e_pec = np.sum(out ** 2)
    e_nr = np.sum(res["nrbc"][0] ** 2)
    assert e_pec >= 0.95 * np.sum(2 * f * f) and e_nr <= 1e-3 * e_pec


def _tet_cavity_error(m):
    vert, tet = wl.kuhn_tet_mesh(m, 0.0, np.random.default_rng(0))
    mesh = go.tet_mesh(vert, tet, bc="pec")
    x, y = mesh.centroid[:, 0], mesh.centroid[:, 1]
    f = np.zeros((6, mesh.ncell))
    f[2] = np.sin(np.pi * x) * np.sin(np.pi * y)
    w = np.pi * math.sqrt(2.0)
    T = 0.3
    dt0 = go.time_step(mesh, 0.4, 1.0)
    nst = int(math.ceil(T / dt0))
    out, info = go.run(mesh, f, np.ones(mesh.ncell), None, 0.4, nst, dt=T / nst)
    ez = np.sin(np.pi * x) * np.sin(np.pi * y) * math.cos(w * T)
    hx = -(np.pi / w) * np.sin(np.pi * x) * np.cos(np.pi * y) * math.sin(w * T)
    hy = (np.pi / w) * np.cos(np.pi * x) * np.sin(np.pi * y) * math.sin(w * T)
    e = np.sqrt(np.sum(mesh.vol * ((out[2] - ez) ** 2 + (out[3] - hx) ** 2 + (out[4] - hy) ** 2)))
    return e, np.max(np.abs(out[[0, 1, 5]]))


def test_tet_pec_cavity_mode_converges():
    """The TM110 mode of the PEC unit cube, E_z = sin(pi x) sin(pi y) cos(w t) with w = pi sqrt2
    and H from Faraday's law, on Kuhn tet meshes with PEC walls: the error at t = 0.3 falls at
    least at first order (Green-Gauss with face averages is first order on tets), and the
    other polarisation (E_x, E_y, H_z), excited only by the mesh's truncation error, shrinks
    with it."""
    e4, o4 = _tet_cavity_error(4)
    e8, o8 = _tet_cavity_error(8)
    assert math.log2(e4 / e8) >= 0.9, (e4, e8)
    assert e8 <= 0.05
    assert o8 <= 0.6 * o4 and o8 <= 0.05, (o4, o8)


# ---------------------------------------------------------------------------- dipole source

def _line_source_field(r, t, I0, w):
    """E_z at distance r of a z-directed line current I(t) = I0 cos(w t) switched on at t = 0 in
    vacuum (c = 1): from d_t^2 E_z - lap E_z = -d_t J_z with the 2-D wave Green's function
    H(t - r) / (2 pi sqrt(t^2 - r^2)), written with tau = r cosh(u):
    E_z = -(1/2 pi) [I0 / sqrt(t^2 - r^2) + int_0^{acosh(t/r)} I'(t - r cosh u) du]."""
    from scipy.integrate import quad
    if t <= r:
        return 0.0
    U = math.acosh(t / r)
    val, _ = quad(lambda u: -I0 * w * math.sin(w * (t - r * math.cosh(u))), 0.0, U, limit=200)
    return -(I0 / math.sqrt(t * t - r * r) + val) / (2.0 * np.pi)


def test_dipole_field_matches_exact_line_source():
    """Sec. 5.4 source J_z = J0 cos(2 pi t / T), T = 0.1, on the 2 x 2 cells around a corner
    (total current I0 = J0 (2h)^2), 80 x 80 cells on [0, 0.4]^2 (20 cells per wavelength): E_z
    at distance ~0.1 follows the exact line-source field within 25% (relative L2 over
    0.15 <= t <= 0.29, before boundary reflections can arrive; the gap is the scheme's phase
    error at 20 cells per wavelength).  A flipped source sign gives ~200%."""
    L, n, T, J0 = 0.4, 80, 0.1, 1.0
    h = L / n
    mesh = go.cartesian_mesh((n, n), (0.0, 0.0), (L, L), ("nrbc",) * 4)
    x, y = mesh.centroid[:, 0], mesh.centroid[:, 1]
    c0 = n // 2
    mask = np.zeros(mesh.ncell)
    for jj in (c0 - 1, c0):
        for ii in (c0 - 1, c0):
            mask[jj * n + ii] = 1.0
    obs = [(c0 + 19) + (c0 - 1) * n, (c0 + 19) + c0 * n]      # symmetric pair about y = L/2
    r = math.hypot(x[obs[0]] - L / 2, y[obs[0]] - L / 2)
    dt = 0.5 * h
    ts, num = [], []

    def cb(k, V):
        ts.append(k * dt)
        num.append(0.5 * (V[obs[0], 2] + V[obs[1], 2]))

    go.run(mesh, np.zeros((3, mesh.ncell)), np.ones(mesh.ncell), None, 0.5, int(0.29 / dt),
           c=1.0, jz_mask=mask, src=(J0, 1.0 / T, 0.0), waveform="cw", callback=cb)
    ts, num = np.array(ts), np.array(num)
    sel = ts >= 0.15
    ex = np.array([_line_source_field(r, t, J0 * (2 * h) ** 2, 2 * np.pi / T) for t in ts[sel]])
    err = np.linalg.norm(num[sel] - ex) / np.linalg.norm(ex)
    assert err <= 0.25, err
    assert np.linalg.norm(-num[sel] - ex) / np.linalg.norm(ex) > 1.5


def test_dipole_workload_mirror_symmetry():
    """The centred dipole (Sec. 5.4) on a square grid: E_z is symmetric under x -> 1 - x,
    y -> 1 - y and x <-> y to rounding (the 2-D scheme and the source are)."""
    w = wl.dipole_tm(n=24, t_end=0.15)
    mesh = go.cartesian_mesh(w.n, w.lo, w.hi, w.bc)
    out, _ = go.run(mesh, w.fields0, w.eps, None, w.cfl, w.steps, jz_mask=w.jz_mask, src=w.src,
                    waveform="cw")
    ez = out[0].reshape(24, 24)                          # [y][x]
    s = np.max(np.abs(ez))
    assert s > 0
    for other in (ez[:, ::-1], ez[::-1, :], ez.T):
        assert np.max(np.abs(ez - other)) <= 1e-12 * s


# ---------------------------------------------------------------------------- divergence cleaning

def test_phm_flux_functions_are_the_cleaning_equations():
    """Sec. 2.1 (PHM system, c = 1, H = B): for a linear field V(x) = V0 + x.G the divergence
    of the fluxes, sum_j F_j(d_j V), must equal -dU/dt of dE/dt = curl H - chi grad phi,
    dH/dt = -curl E - gamma grad psi, dphi/dt = -chi div E, dpsi/dt = -gamma div H, written
    here with curls, gradients and divergences of the derivative matrix."""
    rng = np.random.default_rng(11)
    chi, gamma = 0.7, 1.3
    G = rng.standard_normal((3, 8))                 # G[j] = d_j V
    div_F = sum(go.flux_dir(j, G[j], (chi, gamma)) for j in range(3))
    dE, dH = G[:, 0:3], G[:, 3:6]                   # dE[j, i] = d_j E_i
    curl = lambda d: np.array([d[1, 2] - d[2, 1], d[2, 0] - d[0, 2], d[0, 1] - d[1, 0]])
    grad_phi, grad_psi = G[:, 6], G[:, 7]
    dUdt = np.concatenate([curl(dH) - chi * grad_phi, -curl(dE) - gamma * grad_psi,
                           [-chi * np.trace(dE), -gamma * np.trace(dH)]])
    assert np.allclose(div_F, -dUdt, atol=1e-14)
    # chi = gamma = 0 leaves the Maxwell part and zero cleaning rows
    F0 = go.flux_dir(1, G[1], (0.0, 0.0))
    assert np.allclose(F0[:6], go.flux_dir(1, G[1, :6])) and np.all(F0[6:] == 0.0)


@pytest.mark.parametrize("dim", [2, 3])
def test_phm_equilibrium_compatibility(dim):
    """Sec. 2.2 with the cleaning potentials: sum_k g_k = U, sum_k u_k^j g_k = F_j(V)."""
    rng = np.random.default_rng(12)
    V = rng.standard_normal((30, 8))
    m = np.abs(rng.standard_normal((30, 8))) + 0.5
    m[:, 6:] = 1.0
    phm = (0.6, 1.4)
    for c in (1.5, 2.0):
        u = go.lattice(dim, c)
        g = go.equilibria(m * V, V, u, c, phm)
        assert np.allclose(sum(g), m * V, atol=1e-14, rtol=0)
        for j in range(dim):
            assert np.allclose(sum(u[k, j] * g[k] for k in range(4)), go.flux_dir(j, V, phm),
                               atol=1e-13, rtol=0)


def _cleaning_wave_error(n, dim, speed, potential=None):
    """Standing cleaning wave along x: 2-D (H_x, psi) with gamma, 3-D (E_x, phi) with chi, or in
    3-D with potential="psi" (H_x, psi) with gamma.
    Initial H_x (E_x) = sin(2 pi x); exact H_x = sin(2 pi x) cos(2 pi s t),
    psi = -cos(2 pi x) sin(2 pi s t) (s the cleaning speed)."""
    shape = (n, 4) if dim == 2 else (n, 2, 2)
    h = 1.0 / n
    hi = (1.0, 4 * h) if dim == 2 else (1.0, 2 * h, 2 * h)
    mesh = go.cartesian_mesh(shape, (0.0,) * dim, hi, ("periodic",) * (2 * dim))
    x = mesh.centroid[:, 0]
    if dim == 2:
        f = np.zeros((4, mesh.ncell))
        f[1] = np.sin(2 * np.pi * x)                 # H_x
        phm, a, b = (0.0, speed), 1, 3
    elif potential == "psi":
        f = np.zeros((8, mesh.ncell))
        f[3] = np.sin(2 * np.pi * x)                 # H_x
        phm, a, b = (0.0, speed), 3, 7
    else:
        f = np.zeros((8, mesh.ncell))
        f[0] = np.sin(2 * np.pi * x)                 # E_x
        phm, a, b = (speed, 0.0), 0, 6
    T = 0.4
    cfl = 0.4 if dim == 2 else 0.3
    dt0 = go.time_step(mesh, cfl, 1.0)
    nst = int(math.ceil(T / dt0))
    out, info = go.run(mesh, f, np.ones(mesh.ncell), None, cfl, nst, dt=T / nst, phm=phm)
    w = 2 * np.pi * speed * T
    ea = out[a] - np.sin(2 * np.pi * x) * math.cos(w)
    eb = out[b] + np.cos(2 * np.pi * x) * math.sin(w)
    others = np.delete(out, [a, b], axis=0)
    return math.sqrt(np.mean(ea ** 2 + eb ** 2)), np.max(np.abs(others))


@pytest.mark.parametrize("dim,speed,potential", [(2, 0.5, None), (2, 1.0, None), (3, 0.7, None),
                                                 (3, 0.6, "psi")])
def test_cleaning_wave_second_order(dim, speed, potential):
    """Sec. 2.1: the cleaning potentials carry divergence errors as waves of speed gamma (psi,
    with div B) or chi (phi, with div E).  The 1-D standing wave converges at second order and
    leaves the other components at zero."""
    e1, o1 = _cleaning_wave_error(32, dim, speed, potential)
    e2, o2 = _cleaning_wave_error(64, dim, speed, potential)
    assert math.log2(e1 / e2) >= 1.8, (e1, e2)
    assert e2 <= 2e-3
    assert max(o1, o2) <= 1e-13


def _phm_rho(dim, n, cfl, phm):
    mesh = go.cartesian_mesh((n,) * dim, (0.0,) * dim, (1.0,) * dim, ("periodic",) * (2 * dim))
    m = np.ones((mesh.ncell, 8))
    dt = go.time_step(mesh, cfl)
    C = go.time_coefficients(dt, 0.0)
    comps = [2, 3, 4, 7] if dim == 2 else list(range(8))
    modes = np.array(np.meshgrid(*[np.arange(n)] * dim, indexing="ij")).reshape(dim, -1).T
    rho = 0.0
    for kk in modes:
        k = np.zeros(3)
        k[:dim] = 2 * np.pi * kk
        phase = np.exp(1j * (mesh.centroid @ k))
        Gk = np.zeros((len(comps), len(comps)), dtype=complex)
        for a, ca in enumerate(comps):
            V = np.zeros((mesh.ncell, 8), dtype=complex)
            V[:, ca] = phase
            out = go.step(mesh, V, m, dt, C, phm=phm)
            Gk[:, a] = (out[:, comps] / phase[:, None]).mean(axis=0)
        rho = max(rho, np.abs(np.linalg.eigvals(Gk)).max())
    return rho


@pytest.mark.parametrize("dim,cfl,phm,stable", [
    (2, 0.4, (0.0, 0.5), True), (2, 0.4, (0.0, 1.0), True), (2, 0.5, (0.0, 1.0), False),
    (3, 0.3, (1.0, 1.0), True), (3, 0.4, (1.0, 1.0), False),
])
def test_phm_amplification_spectrum(dim, cfl, phm, stable):
    """Von Neumann stability of the periodic step with cleaning (tau = 0, lattice speed 1):
    with chi, gamma up to 1 the eigenvalues stay in the closed unit disc at CFL 0.4 in 2-D and
    0.3 in 3-D, but not at the Maxwell workloads' CFL (0.5 in 2-D: rho ~ 1.09 at gamma = 1;
    0.4 in 3-D: rho ~ 1.40 at chi = gamma = 1).  Cleaning therefore needs the smaller CFL (or a
    larger lattice speed)."""
    rho = _phm_rho(dim, 8 if dim == 2 else 5, cfl, phm)
    if stable:
        assert rho <= 1.0 + 1e-12, rho
    else:
        assert rho >= 1.05, rho


# ------------------------------------------------------------------------------------------
# Sec. 5.3: slope limiter (van Leer's, a reading: the paper names no limiter)


def test_van_leer_limiter_values():
    """The harmonic mean of same-sign slopes, 0 at an extremum: equal slopes pass unchanged,
    the result lies between the smaller slope and twice it, and it is odd and symmetric."""
    a = np.array([1.0, 1.0, 1.0, 0.0, -2.0, 3.0, -1.0, 0.5])
    b = np.array([1.0, 3.0, -1.0, 2.0, -2.0, 1.0, -3.0, 2.0])
    assert np.array_equal(go.van_leer(a, b), [1.0, 1.5, 0.0, 0.0, -2.0, 1.5, -1.5, 0.8])
    rng = np.random.default_rng(0)
    x, y = rng.standard_normal(1000), rng.standard_normal(1000)
    v = go.van_leer(x, y)
    assert np.array_equal(v, go.van_leer(y, x))
    assert np.array_equal(-v, go.van_leer(-x, -y))
    same = x * y > 0
    lo = np.minimum(np.abs(x), np.abs(y))
    assert np.all(np.abs(v[same]) >= lo[same] * (1 - 1e-15))
    assert np.all(np.abs(v[same]) <= 2 * lo[same] * (1 + 1e-15))
    assert np.all(np.sign(v[same]) == np.sign(x[same]))
    assert np.all(v[~same] == 0.0)


def _vl(a, b):
    return 2 * a * b / (a + b) if a * b > 0 else 0.0


@pytest.mark.parametrize("n,bc", [
    ((5, 4), ("nrbc", "pec", "periodic", "periodic")),
    ((4, 3, 5), ("pec", "nrbc", "nrbc", "pec", "periodic", "periodic")),
])
def test_limited_gradient_brute_force(n, bc):
    """limited_gradient against a per-cell loop over index neighbours: wrap on periodic axes, a
    copy of the cell beyond a non-reflecting side, the PEC mirror image beyond a wall."""
    dim = len(n)
    rng = np.random.default_rng(7)
    h = [0.1 * (d + 1) for d in range(dim)]
    mesh = go.cartesian_mesh(n, (0.0,) * dim, tuple(n[d] * h[d] for d in range(dim)), bc)
    V = rng.standard_normal((mesh.ncell, 6))
    G = go.limited_gradient(mesh, V)
    strides = [1, n[0], n[0] * n[1]][:dim]
    for cell in range(mesh.ncell):
        idx = [(cell // strides[d]) % n[d] for d in range(dim)]
        for d in range(dim):
            nb = []
            for s in (-1, 1):
                j = idx[d] + s
                side = bc[2 * d + (s > 0)]
                if 0 <= j < n[d] or side == "periodic":
                    k = list(idx)
                    k[d] = j % n[d]
                    nb.append(V[sum(k[e] * strides[e] for e in range(dim))])
                elif side == "nrbc":
                    nb.append(V[cell])
                else:
                    e = np.zeros(3)
                    e[d] = 1.0
                    nb.append(go.pec_mirror(e, V[cell]))
            for c in range(6):
                want = _vl((nb[1][c] - V[cell, c]) / h[d], (V[cell, c] - nb[0][c]) / h[d])
                assert abs(G[cell, d, c] - want) <= 1e-12 * max(1.0, abs(want)), (cell, d, c)
        assert np.all(G[cell, dim:] == 0.0)


def test_limited_gradient_exact_on_linear_fields():
    """Away from the boundary a linear field has equal one-sided differences: the limited slope
    is its exact gradient (no clipping in smooth monotone regions)."""
    mesh = go.cartesian_mesh((7, 6, 5), (0.0,) * 3, (0.7, 0.6, 0.5), ("nrbc",) * 6)
    A = np.random.default_rng(2).standard_normal((3, 6))
    V = mesh.centroid @ A + 0.3
    G = go.limited_gradient(mesh, V)
    x = mesh.centroid
    inner = np.all((x > 0.1 + 1e-9) & (x < np.array([0.6, 0.5, 0.4]) - 1e-9), axis=1)
    assert inner.sum() == 5 * 4 * 3
    assert np.allclose(G[inner], np.broadcast_to(A, (inner.sum(), 3, 6)), rtol=0, atol=1e-12)


def _riemann_exact(x, t):
    """Sec. 5.3 states: characteristic variables E_y +- B_z and E_z -+ B_y move at +-1."""
    w1 = np.where(x - t < 0.5, 1.0, -1.0)
    w2 = np.where(x + t < 0.5, 1.0, -1.0)
    w3 = np.where(x - t < 0.5, 0.75, -0.75)
    w4 = np.where(x + t < 0.5, -0.75, 0.75)
    out = np.zeros((6, x.size))
    out[1], out[5] = (w1 + w2) / 2, (w1 - w2) / 2
    out[2], out[4] = (w3 + w4) / 2, (w4 - w3) / 2
    out[3] = 1.0
    return out


def _riemann_run(limiter):
    w = wl.riemann_3d(200, limiter=limiter)
    mesh = go.cartesian_mesh(w.n, w.lo, w.hi, w.bc)
    T = w.extra["t_end"]
    nst = int(math.ceil(T / go.time_step(mesh, w.cfl, 1.0)))
    out, _ = go.run(mesh, w.fields0, w.eps, None, w.cfl, nst, dt=T / nst, limiter=limiter)
    x = w.extra["x"]
    return out, x, _riemann_exact(x, T)


def test_riemann_problem_limiter():
    """Sec. 5.3: with the limiter the Riemann problem is captured without spurious oscillations
    (the characteristic variables overshoot their end states by under 0.2 %); the unlimited
    second-order step overshoots by 10 %.  The L1 error on [0, 1] against the exact two-wave
    solution is 0.013 at the paper's cell size, E_x and B_x stay at their constant values."""
    out, x, ex = _riemann_run("vanleer")
    sel = (x > 0.0) & (x < 1.0)

    def overshoot(o):
        chars = [(o[1] + o[5], 1.0), (o[1] - o[5], 1.0), (o[2] - o[4], 0.75), (o[2] + o[4], 0.75)]
        return max(np.abs(w[sel]).max() - bound for w, bound in chars)

    assert overshoot(out) <= 2e-3, overshoot(out)
    assert np.abs(out - ex)[:, sel].mean() <= 0.0135
    assert np.max(np.abs(out[0])) <= 1e-14 and np.max(np.abs(out[3] - 1.0)) <= 1e-14
    raw, _, _ = _riemann_run(None)
    assert overshoot(raw) >= 0.05, overshoot(raw)


def test_limiter_keeps_second_order_on_smooth_waves():
    """Sec. 5.3: the limited step stays second order in smooth regions: a travelling TM wave
    converges at order >= 1.9 in L1 (the clipping at extrema costs order only in max norm)."""
    errs = []
    for n in (64, 128):
        h = 1.0 / n
        mesh = go.cartesian_mesh((n, 2), (0.0, 0.0), (1.0, 2 * h), ("periodic",) * 4)
        x = mesh.centroid[:, 0]
        f = np.zeros((3, mesh.ncell))
        f[0], f[2] = np.sin(2 * np.pi * x), -np.sin(2 * np.pi * x)    # E_z - H_y moves at +1
        T = 0.5
        nst = int(math.ceil(T / go.time_step(mesh, 0.5, 1.0)))
        out, _ = go.run(mesh, f, np.ones(mesh.ncell), None, 0.5, nst, dt=T / nst,
                        limiter="vanleer")
        errs.append(np.abs(out[0] - np.sin(2 * np.pi * (x - T))).mean())
    assert math.log2(errs[0] / errs[1]) >= 1.9, errs
