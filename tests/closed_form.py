"""Closed form of the GKS interface flux, derived independently of the oracle's per-velocity sums.

Derivation (D3Q4, local frame with normal n and tangents t, w; s_k = u_k / c):
  sum_{k in +} s_k = 2 n, sum_{k in +} s^a s^b = 2 (delta_ab + [ab in {tw, wt}]),
  sum_k s^n s^t s^w = 4, all other third moments vanish.  Hence
  W0   = (U^l + U^r)/2 + (F_n(V^l) - F_n(V^r)) / (2c)
  <u_n g0>            = F_n(V0)
  <u_n u.grad g0>     = c^2 d_n W0 + c (F_w(d_t V0) + F_t(d_w V0))
  <u_n g_t>           = F_n(V0_t),  W0_t = -sum_a F_a(d_a V0)
  free transport      = (F_n^l + F_n^r)/2 - (c/2)(U^r - U^l)
  free transport grad = (c^2/2)(d_n U^l + d_n U^r) + (c/2)(S^l - S^r) + (c/2)(X^l + X^r)
with S = sum_a F_a(d_a V), X = F_w(d_t V) + F_t(d_w V), and X = 0 for D2Q4 (no third moments).
F_e(V) = (-e x H, e x E) is Maxwell's flux along the unit vector e (curl form), written here with
explicit cross products rather than the printed Jacobian blocks.

Works on plain Python numbers (including fractions.Fraction) or numpy arrays per component.
"""
from __future__ import annotations


def cross(a, b):
    return [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]]


def flux_along(e, V):
    """Maxwell flux along direction e of V = (E, H): (-e x H, e x E)."""
    E, H = V[0:3], V[3:6]
    fe = cross(e, H)
    fh = cross(e, E)
    return [-fe[0], -fe[1], -fe[2], fh[0], fh[1], fh[2]]


def add(*vs):
    return [sum(c) for c in zip(*vs)]


def scale(a, v):
    return [a * x for x in v]


def sub(a, b):
    return [x - y for x, y in zip(a, b)]


def mul(m, v):
    return [x * y for x, y in zip(m, v)]


def div(v, m):
    return [x / y for x, y in zip(v, m)]


def dir_deriv(G, e):
    """d_e V = sum_j e_j G[j] for G = [dV/dx, dV/dy, dV/dz] (each a 6-list)."""
    return [G[0][c] * e[0] + G[1][c] * e[1] + G[2][c] * e[2] for c in range(6)]


def face_flux(frame, Vl, Gl, ml, Vr, Gr, mr, ghost, C, dt, c, dim):
    """Flux F.n in the global frame.  frame = (n, t, w) right-handed orthonormal rows (the
    face frame); V 6-lists, G 3 x 6 lists (global derivative directions), m 6-lists (diag M)."""
    n, t, w = frame
    C1, C2, C3, C4, C5 = C
    half = c * 0 + 1
    half = half / 2
    Ul, Ur = mul(ml, Vl), mul(mr, Vr)
    if ghost:
        zero = [0 * x for x in Vl]
        Vr, Ur = zero, zero
        Gr = [zero, zero, zero]
        ms = ml
    else:
        ms = [(a + b) * half for a, b in zip(ml, mr)]
    dirs = (n, t, w)
    dl = [dir_deriv(Gl, e) for e in dirs]      # d_n, d_t, d_w of V^l
    dr = [dir_deriv(Gr, e) for e in dirs]
    Fnl, Fnr = flux_along(n, Vl), flux_along(n, Vr)
    W0 = add(scale(half, add(Ul, Ur)), scale(half / c, sub(Fnl, Fnr)))
    dW0 = [add(scale(half, add(mul(ml, dl[a]), mul(mr, dr[a]))),
               scale(half / c, sub(flux_along(n, dl[a]), flux_along(n, dr[a])))) for a in range(3)]
    V0 = div(W0, ms)
    dV0 = [div(d, ms) for d in dW0]

    def X(d_t, d_w):
        if dim == 2:
            return [0 * x for x in d_t]
        return add(flux_along(w, d_t), flux_along(t, d_w))

    def S(d):
        return add(flux_along(n, d[0]), flux_along(t, d[1]), flux_along(w, d[2]))

    term1 = flux_along(n, V0)
    term2 = add(scale(c * c, dW0[0]), scale(c, X(dV0[1], dV0[2])))
    W0t = scale(-1, S(dV0))
    term3 = flux_along(n, div(W0t, ms))
    term4 = sub(scale(half, add(Fnl, Fnr)), scale(c * half, sub(Ur, Ul)))
    term5 = add(scale(c * c * half, add(mul(ml, dl[0]), mul(mr, dr[0]))),
                scale(c * half, sub(S(dl), S(dr))),
                scale(c * half, add(X(dl[1], dl[2]), X(dr[1], dr[2]))))
    tot = add(scale(C1, term1), scale(C2, term2), scale(C3, term3), scale(C4, term4),
              scale(-C5, term5))
    return scale(1 / dt if not hasattr(dt, "denominator") else 1 / dt, tot)
