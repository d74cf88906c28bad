"""The side-split 3-D face flux (csrc/gks_side3.cuh, generated by paper_2412_16845_gb300/codegen.py)
against the FP64 oracle, on the CPU.

* The committed header is exactly what the generator writes.
* Face by face: F = P^l_L + P^r_R + ie (Q^l_L + Q^r_R) equals the oracle's literal D3Q4 face flux
  of Sec. 3.1 (rotated into T'(n) and back) on x-, y- and z-faces, at several kappa, with random
  states, gradients and permittivities; a non-reflecting face (Sec. 3.1, last paragraph) equals
  the same formula with the ghost's vectors set to zero and ie = 1/eps of the cell, on both the
  low and the high side.
* Whole steps: the CPU emulation of the kernel's arithmetic (tests/side3_emulation.py) equals
  go.step on ragged grids with periodic and non-reflecting sides, unequal cell sizes, random eps
  and a source."""
import os

import numpy as np
import pytest

from oracle import gks_oracle as go
from tests import side3_emulation as emu

sp = pytest.importorskip("sympy")
from paper_2412_16845_gb300 import codegen  # noqa: E402


@pytest.fixture(scope="module")
def terms():
    return codegen.derive()[0]


def test_header_is_generated(terms):
    with open(codegen.HEADER) as f:
        committed = f.read()
    assert committed == codegen.emit(terms), "regenerate: python -m paper_2412_16845_gb300.codegen"


def _oracle_face(A, VL, GL, eL, VR, GR, eR, h, C, dt, ghost):
    """Oracle flux through the face along +e_A between L and R (R ignored for a ghost face),
    times dt / h_A, in global components."""
    n = np.zeros((1, 3))
    n[0, A] = 1.0
    T = go.rotation(n)
    Vl = (VL + 0.5 * h[A] * GL[A])[None]
    Vr = (VR - 0.5 * h[A] * GR[A])[None]
    ml = go.material_diag(np.array([eL]), None)
    mr = go.material_diag(np.array([eR]), None)
    F = go.face_flux_local(go._rot_vec6(T, Vl), go._rot_grad(T, GL[None]), ml,
                           go._rot_vec6(T, Vr), go._rot_grad(T, GR[None]), mr,
                           np.array([ghost]), C, dt, 1.0, 3)
    return go._rot_vec6_back(T, F)[0] * dt / h[A]


def _oracle_low_ghost_face(A, VR, GR, eR, h, C, dt):
    """Oracle flux along +e_A through the low-side non-reflecting face of cell R (outward normal
    -e_A, the cell is the face's l side), times dt / h_A."""
    n = np.zeros((1, 3))
    n[0, A] = -1.0
    T = go.rotation(n)
    Vl = (VR - 0.5 * h[A] * GR[A])[None]
    ml = go.material_diag(np.array([eR]), None)
    F = go.face_flux_local(go._rot_vec6(T, Vl), go._rot_grad(T, GR[None]), ml,
                           go._rot_vec6(T, Vl), go._rot_grad(T, GR[None]), ml,
                           np.array([True]), C, dt, 1.0, 3)
    return -go._rot_vec6_back(T, F)[0] * dt / h[A]


def _cell_inputs(V, G, e, h):
    d = [[2.0 * h[j] * G[j][m] for m in range(6)] for j in range(3)]
    ev = [e * V[m] for m in range(3)]
    ed = [[e * d[j][m] for m in range(3)] for j in range(3)]
    return list(V), d, ev, ed


@pytest.mark.parametrize("kappa", [0.0, 0.05, 1.0, 1e3])
def test_face_flux_matches_oracle(terms, kappa):
    rng = np.random.default_rng(int(kappa * 100) + 7)
    h = (0.05, 0.03, 0.04)
    dt = 0.4 * min(h)
    C = go.time_coefficients(dt, kappa * dt)
    nt = codegen.numeric_terms(terms, C, h, 1.0)
    for trial in range(6):
        VL, VR = rng.standard_normal(6), rng.standard_normal(6)
        GL, GR = rng.standard_normal((3, 6)), rng.standard_normal((3, 6))
        eL, eR = rng.uniform(1.0, 4.0, 2)
        for A in range(3):
            pl, _, ql, _ = emu.side_vectors(nt, A, *_cell_inputs(VL, GL, eL, h))
            _, pr, _, qr = emu.side_vectors(nt, A, *_cell_inputs(VR, GR, eR, h))
            pl, ql, pr, qr = (np.array(x) for x in (pl, ql, pr, qr))
            scale = 1.0 + np.abs(pl).max() + np.abs(pr).max() + np.abs(ql).max()
            ie = 2.0 / (eL + eR)
            ref = _oracle_face(A, VL, GL, eL, VR, GR, eR, h, C, dt, False)
            assert np.abs(pl + pr + ie * (ql + qr) - ref).max() <= 1e-13 * scale, (A, trial)
            # non-reflecting faces: the ghost side contributes nothing, ie = 1/eps of the cell
            ref_hi = _oracle_face(A, VL, GL, eL, VR, GR, eR, h, C, dt, True)
            assert np.abs(pl + ql / eL - ref_hi).max() <= 1e-13 * scale, (A, trial)
            ref_lo = _oracle_low_ghost_face(A, VR, GR, eR, h, C, dt)
            assert np.abs(pr + qr / eR - ref_lo).max() <= 1e-13 * scale, (A, trial)


@pytest.mark.parametrize("n,bc,h", [
    ((6, 5, 4), ("periodic",) * 6, (0.1, 0.1, 0.1)),
    ((7, 4, 5), ("nrbc",) * 6, (0.05, 0.03, 0.04)),
    ((5, 6, 3), ("nrbc", "nrbc", "periodic", "periodic", "nrbc", "nrbc"), (0.04, 0.05, 0.03)),
    ((1, 3, 2), ("periodic", "periodic", "nrbc", "nrbc", "nrbc", "nrbc"), (0.1, 0.1, 0.1)),
])
@pytest.mark.parametrize("kappa", [0.0, 0.05])
def test_step_emulation_matches_oracle(terms, n, bc, h, kappa):
    rng = np.random.default_rng(sum(n) + int(kappa * 100))
    ncell = int(np.prod(n))
    hi = tuple(h[d] * n[d] for d in range(3))
    mesh = go.cartesian_mesh(n, (0.0,) * 3, hi, bc)
    V = rng.standard_normal((ncell, 6))
    eps = rng.uniform(1.0, 3.0, ncell)
    m = go.material_diag(eps, None)
    dt = go.time_step(mesh, 0.4)
    C = go.time_coefficients(dt, kappa * dt)
    jz = np.zeros(ncell)
    jz[rng.choice(ncell, size=2, replace=False)] = rng.uniform(-2, 2, 2)
    ref = go.step(mesh, V, m, dt, C, 1.0, jz)
    nt = codegen.numeric_terms(terms, C, h, 1.0)
    shape = n[::-1]
    out = emu.step(nt, V.T.reshape((6,) + shape), eps.reshape(shape),
                   [bc[2 * j] == "periodic" for j in range(3)], (dt * jz).reshape(shape))
    out = out.reshape(6, ncell).T
    assert np.abs(out - ref).max() <= 1e-13 * (1.0 + np.abs(ref).max())


def test_flux_operation_count():
    """The arithmetic that the 3-D FP32 bound counts: for each axis the generated side split
    spends 66 products (22 multiplications, 44 fused multiply-adds) and 22 additions or
    subtractions on one cell's l- and r-side vectors (both formed from a shared even part and
    an odd part).  Over the three axes that is 264 FP32 operations per cell before the
    differences, the face sums and the update."""
    import re
    with open(codegen.HEADER) as f:
        text = f.read()
    starts = [text.index(f"if constexpr (A == {A})") for A in range(3)]
    ends = starts[1:] + [text.index("\n}\n", starts[2])]
    for A in range(3):
        body = text[starts[A]:ends[A]]
        counts = {op: len(re.findall(r"OP::%s\(" % op, body)) for op in ("mul", "fma", "add", "sub")}
        assert counts == {"mul": 22, "fma": 44, "add": 11, "sub": 11}, (A, counts)
