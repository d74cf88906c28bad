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


def main(argv=None) -> int:
    terms, _ = derive()
    text = emit(terms)
    with open(HEADER, "w") as f:
        f.write(text)
    n = [sum(len(v) for v in terms[A].values()) for A in range(3)]
    print(f"wrote {HEADER}: terms per axis {n}")
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
