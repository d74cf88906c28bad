"""Code generator for the side-split GKS face flux of the 3-D Cartesian step kernel.

Writes ``csrc/gks_side3.cuh``.  Run ``python -m paper_2412_16845_gb300.codegen`` (needs sympy)
after changing it; the build compiles the committed header and does not run this module, and a
CPU test checks that the committed header is what this module produces.

What it derives (Sec. 3.1, Sec. 2.2).  With mu = 1 the time-integrated flux through a face of a
Cartesian grid is linear in the reconstructed states and gradients of its two cells.  Its
coefficients depend on the cells' permittivities only through U = M V (eps on the E rows of each
side) and through the interface material M_s = (M_l + M_r)/2, whose inverse enters V0 = W0/M_s
and V0_t = W0_t/M_s exactly once in every term.  So the flux splits into parts owned by one side:

    F = P^l + P^r + ie (Q^l + Q^r),        ie = 2 / (eps_l + eps_r),

where P^s and Q^s are linear in the data of side s alone (its V, its raw central differences
and the eps-weighted E rows of both).  A cell is the l side of its face at +1/2 and the r side
of its face at -1/2 along every axis, and its reconstructions V +- (h/2) d_n V differ only in
sign, so the generator also splits P and Q into the part Ev that both faces share and the part Od
that changes sign (P^l = Ev + Od, P^r = Ev - Od).  Each cell then computes 66 products per axis
and sends 12 numbers to its neighbour instead of its whole state and gradient.

The flux itself is formed here from the D3Q4 sums of Sec. 3.1 (equilibria, upwind half-sums,
interface equilibrium and its gradient, compatibility time derivative, the five C-terms),
symbolically, in the face frame T'(n) of each axis; no closed form is assumed.  A non-reflecting
face (Sec. 3.1, last paragraph) is the same formula with the ghost side's P and Q set to zero and
ie = 1/eps of the cell, which the CPU tests check against the oracle's literal ghost face.
"""
from __future__ import annotations

import os
import sys

HEADER = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc", "gks_side3.cuh")

# Face frames T'(n) of Sec. 3.1 for n = +e_x, +e_y, +e_z: rows are the local axes (n, t, w) in
# global coordinates.  They are the printed T'(n) at these normals (signed permutations).
FRAMES = (
    ((1, 0, 0), (0, 1, 0), (0, 0, 1)),
    ((0, 1, 0), (-1, 0, 0), (0, 0, 1)),
    ((0, 0, 1), (0, 1, 0), (-1, 0, 0)),
)
COMP = ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz")


def _local_flux(sp):
    """The face flux in the face frame as sympy expressions of both sides' data.

    Returns (F, syms) with F[m] the flux component m (times dt / h_n: the K_i are C_i / h_n)
    and syms the side symbols: V_s[m] (reconstructed state), D_s[a][m] (derivative along local
    axis a), eps_s; mu = 1."""
    c = sp.Symbol("c", positive=True)
    K = sp.symbols("K1:6")
    el, er = sp.symbols("eps_l eps_r", positive=True)

    def flux_dir(j, V):                       # F_j(V) of Sec. 2.1 acting on (E, H)
        M = (((0, 0, 0), (0, 0, 1), (0, -1, 0)),
             ((0, 0, -1), (0, 0, 0), (1, 0, 0)),
             ((0, 1, 0), (-1, 0, 0), (0, 0, 0)))[j]
        E, H = V[:3], V[3:]
        return ([sum(M[a][b] * H[b] for b in range(3)) for a in range(3)] +
                [sum(M[b][a] * E[b] for b in range(3)) for a in range(3)])

    u = [[c * s for s in k] for k in ((1, 1, 1), (1, -1, -1), (-1, 1, -1), (-1, -1, 1))]

    def equilibria(U, V):                     # g_k = U/4 + u_k . F(V) / (4 c^2)  (Sec. 2.2)
        F = [flux_dir(j, V) for j in range(3)]
        return [[U[m] / 4 + sum(uk[j] * F[j][m] for j in range(3)) / (4 * c * c)
                 for m in range(6)] for uk in u]

    def side(tag):
        V = list(sp.symbols(f"{tag}V0:6"))
        D = [list(sp.symbols(f"{tag}D{a}_0:6")) for a in range(3)]
        return V, D

    lV, lD = side("l")
    rV, rD = side("r")
    ml = [el] * 3 + [1] * 3
    mr = [er] * 3 + [1] * 3
    gl = equilibria([ml[m] * lV[m] for m in range(6)], lV)
    gr = equilibria([mr[m] * rV[m] for m in range(6)], rV)
    dgl = [equilibria([ml[m] * lD[j][m] for m in range(6)], lD[j]) for j in range(3)]
    dgr = [equilibria([mr[m] * rD[j][m] for m in range(6)], rD[j]) for j in range(3)]
    pos, neg = (0, 1), (2, 3)                 # u_k . n > 0 (l side) and < 0 (r side)
    W0 = [sum(gl[k][m] for k in pos) + sum(gr[k][m] for k in neg) for m in range(6)]
    dW0 = [[sum(dgl[j][k][m] for k in pos) + sum(dgr[j][k][m] for k in neg) for m in range(6)]
           for j in range(3)]
    ms = [(ml[m] + mr[m]) / 2 for m in range(6)]
    V0 = [W0[m] / ms[m] for m in range(6)]
    dV0 = [[dW0[j][m] / ms[m] for m in range(6)] for j in range(3)]
    g0 = equilibria(W0, V0)
    dg0 = [equilibria(dW0[j], dV0[j]) for j in range(3)]
    W0t = [-sum(u[k][j] * dg0[j][k][m] for k in range(4) for j in range(3)) for m in range(6)]
    gt = equilibria(W0t, [W0t[m] / ms[m] for m in range(6)])

    def udg(dg, k, m):
        return sum(u[k][j] * dg[j][k][m] for j in range(3))

    T1 = [sum(u[k][0] * g0[k][m] for k in range(4)) for m in range(6)]
    T2 = [sum(u[k][0] * udg(dg0, k, m) for k in range(4)) for m in range(6)]
    T3 = [sum(u[k][0] * gt[k][m] for k in range(4)) for m in range(6)]
    T4 = [sum(u[k][0] * gl[k][m] for k in pos) + sum(u[k][0] * gr[k][m] for k in neg)
          for m in range(6)]
    T5 = [sum(u[k][0] * udg(dgl, k, m) for k in pos) + sum(u[k][0] * udg(dgr, k, m) for k in neg)
          for m in range(6)]
    F = [sp.expand(K[0] * T1[m] + K[1] * T2[m] + K[2] * T3[m] + K[3] * T4[m] - K[4] * T5[m])
         for m in range(6)]
    return F, dict(c=c, K=K, el=el, er=er, lV=lV, lD=lD, rV=rV, rD=rD)


def _split_coefficient(sp, coef, es, el, er):
    """coef(eps_l, eps_r) = a + b ie + g eps_s + d eps_s ie with ie = 2/(eps_l + eps_r)."""
    a, b, g, d = sp.symbols("_a _b _g _d")
    expr = sp.together(coef - (a + b * 2 / (el + er) + g * es + d * es * 2 / (el + er)))
    eqs = sp.Poly(sp.expand(sp.numer(expr)), el, er).coeffs()
    sol = sp.solve(eqs, [a, b, g, d], dict=True)
    if not sol:
        raise RuntimeError(f"coefficient {coef} does not split")
    return [sp.nsimplify(sp.simplify(sol[0].get(s, 0)), rational=True) for s in (a, b, g, d)]


def derive():
    """Per axis A: the terms of Ev/Od of P and Q in global components.

    Returns (terms, syms): terms[A][(part, m)] = list of (coefficient expression, input name),
    part in ('EvP', 'OdP', 'EvQ', 'OdQ'), m the global component; inputs are 'v{m}' (cell state),
    'd{j}_{m}' (raw central difference V_{+1} - V_{-1} along global axis j), 'ev{m}' (eps E_m)
    and 'ed{j}_{m}' (eps times d{j}_{m}, m < 3).  Coefficients use K1..K5 = C_i / h_A, c and
    ih{j} = 1 / (2 h_j)."""
    import sympy as sp

    F, s = _local_flux(sp)
    c, el, er = s["c"], s["el"], s["er"]
    ih = sp.symbols("ih0:3", positive=True)
    # per local input: [a, b, g, d] for each output component, per side
    split = {}
    for m in range(6):
        for side, V, D, es in (("l", s["lV"], s["lD"], el), ("r", s["rV"], s["rD"], er)):
            for name, x in [(f"V{k}", V[k]) for k in range(6)] + \
                    [(f"D{a}_{k}", D[a][k]) for a in range(3) for k in range(6)]:
                coef = F[m].coeff(x)
                if coef != 0:
                    split[(m, side, name)] = _split_coefficient(sp, coef, es, el, er)
    terms = []
    for A, T in enumerate(FRAMES):
        T6 = [[0] * 6 for _ in range(6)]
        for a in range(3):
            for j in range(3):
                T6[a][j] = T[a][j]
                T6[3 + a][3 + j] = T[a][j]
        # global inputs as symbols
        v = sp.symbols("v0:6")
        d = [sp.symbols(f"d{j}_0:6") for j in range(3)]
        ev = sp.symbols("ev0:3")
        ed = [sp.symbols(f"ed{j}_0:3") for j in range(3)]

        def glob(k, j, weighted):
            """Local derivative/value of component k along local axis j (j = None: the value),
            in global inputs (true derivatives: raw difference times ih)."""
            out = 0
            for kk in range(6):
                t = T6[k][kk]
                if t == 0:
                    continue
                if j is None:
                    src = (ev[kk] if weighted else v[kk])
                else:
                    src = sum(T[j][jj] * ih[jj] * (ed[jj][kk] if weighted else d[jj][kk])
                              for jj in range(3) if T[j][jj] != 0)
                out += t * src
            return out

        hn = 1 / (2 * ih[A])
        P = {"l": [0] * 6, "r": [0] * 6}
        Q = {"l": [0] * 6, "r": [0] * 6}
        for (m, side, name), (al, be, ga, de) in split.items():
            sgn = 1 if side == "l" else -1          # reconstruction V +- (h/2) d_n V
            if name.startswith("V"):
                k = int(name[1:])
                x = glob(k, None, False) + sgn * hn / 2 * glob(k, 0, False)
                ex = glob(k, None, True) + sgn * hn / 2 * glob(k, 0, True) if k < 3 else 0
            else:
                a, k = int(name[1]), int(name[3:])
                x = glob(k, a, False)
                ex = glob(k, a, True) if k < 3 else 0
            P[side][m] += al * x + ga * ex
            Q[side][m] += be * x + de * ex
        # back to global components: F_glob = T6^T F_loc
        inputs = list(v) + [x for row in d for x in row] + list(ev) + [x for row in ed for x in row]
        out = {}
        for part, (Xl, Xr, sg) in (("EvP", (P["l"], P["r"], 1)), ("OdP", (P["l"], P["r"], -1)),
                                   ("EvQ", (Q["l"], Q["r"], 1)), ("OdQ", (Q["l"], Q["r"], -1))):
            for mg in range(6):
                e = sum(T6[ml][mg] * (Xl[ml] + sg * Xr[ml]) / 2 for ml in range(6))
                e = sp.expand(e)
                lst = []
                for x in inputs:
                    cf = sp.factor(sp.simplify(e.coeff(x)))
                    if cf != 0:
                        lst.append((cf, str(x)))
                out[(part, mg)] = lst
        terms.append(out)
    return terms, dict(c=c, ih=ih)


# ------------------------------------------------------------------------------- emission
def _cexpr(sp, e):
    """C++ expression of a coefficient (double arithmetic)."""
    code = sp.ccode(sp.nsimplify(e))
    return code.replace("pow(", "std::pow(")


def _input_ref(name):
    if name.startswith("v"):
        return f"v[{name[1:]}]"
    if name.startswith("ev"):
        return f"ev[{name[2:]}]"
    if name.startswith("ed"):
        j, m = name[2:].split("_")
        return f"ed[{j}][{m}]"
    j, m = name[1:].split("_")
    return f"d[{j}][{m}]"


def emit(terms) -> str:
    import sympy as sp

    lines = []
    w = lines.append
    w("// GENERATED by paper_2412_16845_gb300/codegen.py from the D3Q4 sums of Sec. 3.1; do not")
    w("// edit by hand (regenerate with `python -m paper_2412_16845_gb300.codegen`).")
    w("//")
    w("// Side-split face flux of the 3-D Cartesian step with mu = 1.  The flux through the face")
    w("// between cells L and R along axis A (global components, times dt/h_A) is")
    w("//     F = (Ev_L + Od_L) + (Ev_R - Od_R) + ie [(EvQ_L + OdQ_L) + (EvQ_R - OdQ_R)],")
    w("//     ie = 2 / (eps_L + eps_R),")
    w("// where Ev, Od, EvQ, OdQ of a cell are linear in its state v, its raw central differences")
    w("// d[j] = V(+e_j) - V(-e_j) and the eps-weighted E rows ev = eps E, ed[j] = eps d[j] (E")
    w("// rows).  A non-reflecting face takes zero for the ghost's four vectors and ie = 1/eps of")
    w("// the cell.")
    w("#pragma once")
    w("")
    w("#include <cmath>")
    w("")
    w("namespace gks {")
    w("")
    slots = []
    index = {}
    for A in range(3):
        for key in sorted(terms[A]):
            for cf, _ in terms[A][key]:
                k = (A, sp.srepr(cf))
                if k not in index:
                    index[k] = len([s for s in slots if s[0] == A])
                    slots.append((A, cf))
    nk = max(sum(1 for s in slots if s[0] == A) for A in range(3))
    w(f"constexpr int kSide3K = {nk};   // coefficient slots per axis")
    w("")
    w("// Coefficient slots of axis A (0 = x, 1 = y, 2 = z) from C1..C5 of Sec. 3.1, the cell")
    w("// sizes h[3] and the lattice speed c.  Unused slots are zero.")
    w("inline void side3_coefficients(const double C[5], const double h[3], double c, int A,")
    w("                               double k[kSide3K]) {")
    w("  const double K1 = C[0] / h[A], K2 = C[1] / h[A], K3 = C[2] / h[A], K4 = C[3] / h[A],")
    w("               K5 = C[4] / h[A];")
    w("  const double ih0 = 0.5 / h[0], ih1 = 0.5 / h[1], ih2 = 0.5 / h[2];")
    w("  (void)K1; (void)K2; (void)K3; (void)K4; (void)K5; (void)ih0; (void)ih1; (void)ih2;")
    w("  for (int i = 0; i < kSide3K; ++i) k[i] = 0.0;")
    for A in range(3):
        w(f"  if (A == {A}) {{")
        for (AA, cf) in slots:
            if AA != A:
                continue
            w(f"    k[{index[(A, sp.srepr(cf))]}] = {_cexpr(sp, cf)};")
        w("  }")
    w("}")
    w("")
    w("// Ev, Od, EvQ, OdQ of one cell for faces along axis A, returned as the cell's l-side")
    w("// vectors (pl, ql: its face at +1/2) and r-side vectors (pr, qr: its face at -1/2).")
    w("// OP supplies mul(k, x), fma(k, x, acc), add, sub for the value type T (a scalar or a")
    w("// pair of cells); k holds the slots of axis A in the form OP expects.")
    w("template <int A, class OP, class T, class KT>")
    w("__device__ __forceinline__ void side3(const T v[6], const T d[3][6], const T ev[3],")
    w("                                      const T ed[3][3], const KT *k, T pl[6], T pr[6],")
    w("                                      T ql[6], T qr[6]) {")
    for A in range(3):
        w(f"  if constexpr (A == {A}) {{")
        for m in range(6):
            for part in ("EvP", "OdP", "EvQ", "OdQ"):
                lst = terms[A][(part, m)]
                var = f"{part.lower()}{m}"
                if not lst:
                    continue
                first = True
                for cf, x in lst:
                    ks = f"k[{index[(A, sp.srepr(cf))]}]"
                    if first:
                        w(f"    T {var} = OP::mul({ks}, {_input_ref(x)});")
                        first = False
                    else:
                        w(f"    {var} = OP::fma({ks}, {_input_ref(x)}, {var});")
            for P, l, r in (("P", "pl", "pr"), ("Q", "ql", "qr")):
                ev = terms[A][("Ev" + P, m)]
                od = terms[A][("Od" + P, m)]
                e, o = f"ev{P.lower()}{m}", f"od{P.lower()}{m}"
                if ev and od:
                    w(f"    {l}[{m}] = OP::add({e}, {o}); {r}[{m}] = OP::sub({e}, {o});")
                elif ev:
                    w(f"    {l}[{m}] = {e}; {r}[{m}] = {e};")
                elif od:
                    w(f"    {l}[{m}] = {o}; {r}[{m}] = OP::neg({o});")
                else:
                    w(f"    {l}[{m}] = OP::zero(); {r}[{m}] = OP::zero();")
        w("  }")
    w("}")
    w("")
    w("}  // namespace gks")
    return "\n".join(lines) + "\n"


def numeric_terms(terms, C, h, c):
    """The term lists with numeric coefficients (float) for given C1..C5, h[3] and c: for the
    CPU emulation of the kernel's arithmetic in the tests."""
    import sympy as sp

    K = sp.symbols("K1:6")
    ih = sp.symbols("ih0:3", positive=True)
    cs = sp.Symbol("c", positive=True)
    out = []
    for A in range(3):
        sub = {K[i]: C[i] / h[A] for i in range(5)}
        sub.update({ih[j]: 0.5 / h[j] for j in range(3)})
        sub[cs] = c
        out.append({key: [(float(cf.subs(sub)), x) for cf, x in lst]
                    for key, lst in terms[A].items()})
    return out


# ==================================================================== divergence-cleaning flux
# The same construction for the cleaning system of Sec. 2.1 (V = (E, H, phi, psi), fluxes with
# chi and gamma) in the face frame of an arbitrary face: the folded interior-face flux with
# mu = 1 (flux3_phm_mu1) that the 3-D cleaning kernel evaluates, written to csrc/gks_phm3.cuh.
PHM_HEADER = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc", "gks_phm3.cuh")
PHM_COMP = ("En", "Et", "Ew", "Hn", "Ht", "Hw", "Ph", "Ps")
PHM_FIELDS = (("v", "v"), ("n", "dn"), ("t", "dt"), ("w", "dw"))   # input tag, Side8 member


def _local_flux_phm(sp):
    """The cleaning system's face flux in the face frame (normal = local axis 0) as sympy
    expressions: F[m] times dt / h (K_i = C_i / h), inputs per side s: V_s[m] (reconstructed
    value) and D_s[a][m] (derivative along local axis a = n, t, w), permittivity eps_s, mu = 1."""
    c = sp.Symbol("c", positive=True)
    chi, gam = sp.symbols("chi gam", positive=True)
    K = sp.symbols("K1:6")
    el, er = sp.symbols("eps_l eps_r", positive=True)
    blocks = (((0, 0, 0), (0, 0, 1), (0, -1, 0)),
              ((0, 0, -1), (0, 0, 0), (1, 0, 0)),
              ((0, 1, 0), (-1, 0, 0), (0, 0, 0)))

    def flux_dir(j, V):                       # F_j of Sec. 2.1 with the cleaning terms
        M = blocks[j]
        E, H, ph, ps = V[:3], V[3:6], V[6], V[7]
        out = ([sum(M[a][b] * H[b] for b in range(3)) for a in range(3)] +
               [sum(M[b][a] * E[b] for b in range(3)) for a in range(3)] + [0, 0])
        out[j] += chi * ph
        out[3 + j] += gam * ps
        out[6] = chi * E[j]
        out[7] = gam * H[j]
        return out

    u = [[c * s for s in k] for k in ((1, 1, 1), (1, -1, -1), (-1, 1, -1), (-1, -1, 1))]

    def equilibria(U, V):                     # g_k = U/4 + u_k . F(V) / (4 c^2)  (Sec. 2.2)
        F = [flux_dir(j, V) for j in range(3)]
        return [[U[m] / 4 + sum(uk[j] * F[j][m] for j in range(3)) / (4 * c * c)
                 for m in range(8)] for uk in u]

    def side(tag):
        return (list(sp.symbols(f"{tag}V0:8")),
                [list(sp.symbols(f"{tag}D{a}_0:8")) for a in range(3)])

    lV, lD = side("l")
    rV, rD = side("r")
    ml = [el] * 3 + [1] * 5
    mr = [er] * 3 + [1] * 5
    gl = equilibria([ml[m] * lV[m] for m in range(8)], lV)
    gr = equilibria([mr[m] * rV[m] for m in range(8)], rV)
    dgl = [equilibria([ml[m] * lD[j][m] for m in range(8)], lD[j]) for j in range(3)]
    dgr = [equilibria([mr[m] * rD[j][m] for m in range(8)], rD[j]) for j in range(3)]
    pos, neg = (0, 1), (2, 3)
    W0 = [sum(gl[k][m] for k in pos) + sum(gr[k][m] for k in neg) for m in range(8)]
    dW0 = [[sum(dgl[j][k][m] for k in pos) + sum(dgr[j][k][m] for k in neg) for m in range(8)]
           for j in range(3)]
    ms = [(ml[m] + mr[m]) / 2 for m in range(8)]
    V0 = [W0[m] / ms[m] for m in range(8)]
    dV0 = [[dW0[j][m] / ms[m] for m in range(8)] for j in range(3)]
    g0 = equilibria(W0, V0)
    dg0 = [equilibria(dW0[j], dV0[j]) for j in range(3)]
    W0t = [-sum(u[k][j] * dg0[j][k][m] for k in range(4) for j in range(3)) for m in range(8)]
    gt = equilibria(W0t, [W0t[m] / ms[m] for m in range(8)])

    def udg(dg, k, m):
        return sum(u[k][j] * dg[j][k][m] for j in range(3))

    T1 = [sum(u[k][0] * g0[k][m] for k in range(4)) for m in range(8)]
    T2 = [sum(u[k][0] * udg(dg0, k, m) for k in range(4)) for m in range(8)]
    T3 = [sum(u[k][0] * gt[k][m] for k in range(4)) for m in range(8)]
    T4 = [sum(u[k][0] * gl[k][m] for k in pos) + sum(u[k][0] * gr[k][m] for k in neg)
          for m in range(8)]
    T5 = [sum(u[k][0] * udg(dgl, k, m) for k in pos) + sum(u[k][0] * udg(dgr, k, m) for k in neg)
          for m in range(8)]
    F = [sp.expand(K[0] * T1[m] + K[1] * T2[m] + K[2] * T3[m] + K[3] * T4[m] - K[4] * T5[m])
         for m in range(8)]
    return F, dict(c=c, chi=chi, gam=gam, K=K, el=el, er=er, lV=lV, lD=lD, rV=rV, rD=rD)


def derive_phm():
    """The folded interior-face cleaning flux with mu = 1: per output component m (local frame)
    the list of terms (group, tag, k, A, B), each (A + B ie) group(tag_k), ie = 2/(eps_l +
    eps_r), with group S = x_l + x_r, D = x_r - x_l, SE = eps_l x_l + eps_r x_r or
    DE = eps_r x_r - eps_l x_l of input x = value (tag v) or derivative along n, t, w of
    component k.  A and B are polynomials in K1..K5 = C_i / h, c, chi and gam."""
    import sympy as sp

    F, s = _local_flux_phm(sp)
    el, er = s["el"], s["er"]
    out = []
    for m in range(8):
        terms = []
        for fi, (tag, _) in enumerate(PHM_FIELDS):
            for k in range(8):
                xl = s["lV"][k] if tag == "v" else s["lD"][fi - 1][k]
                xr = s["rV"][k] if tag == "v" else s["rD"][fi - 1][k]
                cl, cr = F[m].coeff(xl), F[m].coeff(xr)
                zero = [sp.Integer(0)] * 4
                al, bl, gl, dl = zero if cl == 0 else _split_coefficient(sp, cl, el, el, er)
                ar, br, gr, dr = zero if cr == 0 else _split_coefficient(sp, cr, er, el, er)
                for grp, A, B in (("S", (al + ar) / 2, (bl + br) / 2),
                                  ("D", (ar - al) / 2, (br - bl) / 2),
                                  ("SE", (gl + gr) / 2, (dl + dr) / 2),
                                  ("DE", (gr - gl) / 2, (dr - dl) / 2)):
                    A, B = sp.factor(sp.expand(A)), sp.factor(sp.expand(B))
                    if A != 0 or B != 0:
                        terms.append((grp, tag, k, A, B))
        out.append(terms)
    return out


def _phm_slots(sp, terms):
    """Coefficient slots of the folded flux: constants k[] (B = 0) and pairs (a[], b[]) for the
    ie-dependent coefficients, shared between terms up to sign.  Returns (kslots, pslots, ref)
    with ref[(m, i)] = (sign, kind, slot) for term i of component m."""
    kslots, pslots, kidx, pidx, ref = [], [], {}, {}, {}
    for m, lst in enumerate(terms):
        for i, (_, _, _, A, B) in enumerate(lst):
            if B == 0:
                key, neg = sp.srepr(A), sp.srepr(sp.factor(-A))
                if key in kidx:
                    ref[(m, i)] = (1, "k", kidx[key])
                elif neg in kidx:
                    ref[(m, i)] = (-1, "k", kidx[neg])
                else:
                    kidx[key] = len(kslots)
                    kslots.append(A)
                    ref[(m, i)] = (1, "k", kidx[key])
            else:
                key = (sp.srepr(A), sp.srepr(B))
                neg = (sp.srepr(sp.factor(-A)), sp.srepr(sp.factor(-B)))
                if key in pidx:
                    ref[(m, i)] = (1, "c", pidx[key])
                elif neg in pidx:
                    ref[(m, i)] = (-1, "c", pidx[neg])
                else:
                    pidx[key] = len(pslots)
                    pslots.append((A, B))
                    ref[(m, i)] = (1, "c", pidx[key])
    return kslots, pslots, ref


def _group_name(grp, tag, k):
    return f"{grp}_{tag}{PHM_COMP[k]}"


def _group_expr(grp, tag, k):
    mem = dict(PHM_FIELDS)[tag]
    x_l, x_r = f"l.{mem}[{k}]", f"r.{mem}[{k}]"
    return {"S": f"{x_l} + {x_r}", "D": f"{x_r} - {x_l}",
            "SE": f"el * {x_l} + er * {x_r}", "DE": f"er * {x_r} - el * {x_l}"}[grp]


def emit_phm(terms) -> str:
    import sympy as sp

    kslots, pslots, ref = _phm_slots(sp, terms)
    lines = []
    w = lines.append
    w("// GENERATED by paper_2412_16845_gb300/codegen.py from the D3Q4 sums of Sec. 3.1 for the")
    w("// divergence-cleaning system of Sec. 2.1; do not edit by hand (regenerate with")
    w("// `python -m paper_2412_16845_gb300.codegen`).")
    w("//")
    w("// Interior-face flux of the cleaning system with mu = 1 in the face frame (components En,")
    w("// Et, Ew, Hn, Ht, Hw, phi, psi; times dt/h), folded: every term is a coefficient times a")
    w("// sum S(x) = x_l + x_r, a difference D(x) = x_r - x_l or their eps-weighted forms")
    w("// SE(x) = eps_l x_l + eps_r x_r, DE(x) = eps_r x_r - eps_l x_l of one side quantity x")
    w("// (reconstructed value v, derivative along n, t or w).  A coefficient is a constant k[] or")
    w("// a[] + b[] ie with ie = 2/(eps_l + eps_r), both polynomials in C_i/h, c, chi and gamma")
    w("// folded on the host.  Included by gks_flux3.cuh after Side8.")
    w("#pragma once")
    w("")
    w("#include <cmath>")
    w("")
    w("namespace gks {")
    w("")
    w("template <typename T>")
    w("struct F8K {")
    w(f"  T k[{len(kslots)}];")
    w(f"  T a[{len(pslots)}], b[{len(pslots)}];")
    w("};")
    w("")
    w("template <typename T>")
    w("inline F8K<T> make_f8k(const double C[5], double h, double c, double chi, double gam) {")
    w("  const double K1 = C[0] / h, K2 = C[1] / h, K3 = C[2] / h, K4 = C[3] / h, K5 = C[4] / h;")
    w("  (void)K1; (void)K2; (void)K3; (void)K4; (void)K5; (void)chi; (void)gam;")
    w("  F8K<T> f;")
    for i, A in enumerate(kslots):
        w(f"  f.k[{i}] = T({_cexpr(sp, A)});")
    for i, (A, B) in enumerate(pslots):
        w(f"  f.a[{i}] = T({_cexpr(sp, A)});")
        w(f"  f.b[{i}] = T({_cexpr(sp, B)});")
    w("  return f;")
    w("}")
    w("")
    w("template <typename T>")
    w("__device__ __forceinline__ void flux3_phm_mu1(const Side8<T> &l, const Side8<T> &r,")
    w("                                              const F8K<T> &K, T ie, T out[8]) {")
    w("  const T el = l.eps, er = r.eps;")
    w("  (void)el; (void)er;")
    groups = sorted({(g, t, k) for lst in terms for (g, t, k, _, _) in lst},
                    key=lambda x: (x[0], x[1], x[2]))
    for g, t, k in groups:
        w(f"  const T {_group_name(g, t, k)} = {_group_expr(g, t, k)};")
    used = sorted({ref[(m, i)][2] for m, lst in enumerate(terms) for i in range(len(lst))
                   if ref[(m, i)][1] == "c"})
    for j in used:
        A, _ = pslots[j]
        w(f"  const T c{j} = " + (f"K.b[{j}] * ie;" if A == 0 else f"K.a[{j}] + K.b[{j}] * ie;"))
    for m, lst in enumerate(terms):
        parts = []
        for i, (g, t, k, _, _) in enumerate(lst):
            sgn, kind, slot = ref[(m, i)]
            coef = f"K.k[{slot}]" if kind == "k" else f"c{slot}"
            op = ("-" if sgn < 0 else "") if not parts else (" - " if sgn < 0 else " + ")
            parts.append(f"{op}{coef} * {_group_name(g, t, k)}")
        body = "".join(parts) if parts else "T(0)"
        w(f"  out[{m}] = {body};")
    w("}")
    w("")
    w("}  // namespace gks")
    return "\n".join(lines) + "\n"


def phm_numeric(terms, C, h, c, chi, gam):
    """The folded cleaning flux with numeric coefficients, as the header evaluates it: returns
    f(l, r) for sides given as dicts of arrays v, dn, dt, dw ([8]) and eps (for the CPU tests)."""
    import sympy as sp

    K = sp.symbols("K1:6")
    sub = {K[i]: C[i] / h for i in range(5)}
    sub.update({sp.Symbol("c", positive=True): c, sp.Symbol("chi", positive=True): chi,
                sp.Symbol("gam", positive=True): gam})
    num = [[(g, dict(PHM_FIELDS)[t], k, float(sp.sympify(A).subs(sub)),
             float(sp.sympify(B).subs(sub))) for (g, t, k, A, B) in lst] for lst in terms]

    def flux(l, r):
        ie = 2.0 / (l["eps"] + r["eps"])
        el, er = l["eps"], r["eps"]
        out = []
        for lst in num:
            acc = 0.0
            for g, mem, k, a, b in lst:
                xl, xr = l[mem][k], r[mem][k]
                x = {"S": xl + xr, "D": xr - xl, "SE": el * xl + er * xr,
                     "DE": er * xr - el * xl}[g]
                acc = acc + (a + b * ie) * x
            out.append(acc)
        return out
    return flux


def main(argv=None) -> int:
    terms, _ = derive()
    text = emit(terms)
    with open(HEADER, "w") as f:
        f.write(text)
    n = [sum(len(v) for v in terms[A].values()) for A in range(3)]
    print(f"wrote {HEADER}: terms per axis {n}")
    pterms = derive_phm()
    with open(PHM_HEADER, "w") as f:
        f.write(emit_phm(pterms))
    print(f"wrote {PHM_HEADER}: terms per component {[len(t) for t in pterms]}")
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
