"""Pins for the oracle's element matrices and stabilisation constant.

* Q1 stiffness / mass of a whole cell: textbook closed forms, and the 9-point
  node stencil 8/3, -1/3 they give in 2D.
* A straight (vertical) cut reduces to the 1D ghost-FEM system printed in
  Sec. 4 (Eq. ls1dA, Eq. ls1dF) tensored with 1D Q1 factors in y: this pins
  the Nitsche signs and the normal orientation.
* Eq. c_triangle against the generalized-eigenvalue definition (Sec. 5.2).
* Quadrilateral with equal cut lengths: C = 1/(theta h) (Sec. 5.3, rectangle
  test; Sec. 4.4 1D value).
* Eq. c_pentagon = Eq. c_triangle at theta1 = theta2 = 1, and it bounds the
  definition for pentagons and hexagons (so lambda = gamma C stays coercive).
"""
import math

import numpy as np
import pytest

from oracle import ghostfem as gf
from paper_2505_05105_gb300 import workloads as wl


def test_interior_q1_matrices_closed_form():
    h = 0.037
    S, M = gf.interior_cell_matrices(h)
    S_ref = np.array([[4, -1, -1, -2], [-1, 4, -2, -1], [-1, -2, 4, -1], [-2, -1, -1, 4]]) / 6.0
    M_ref = np.array([[4, 2, 2, 1], [2, 4, 1, 2], [2, 1, 4, 2], [1, 2, 2, 4]]) * h * h / 36.0
    np.testing.assert_allclose(S, S_ref, rtol=0, atol=1e-14)
    np.testing.assert_allclose(M, M_ref, rtol=1e-13, atol=0)


def test_interior_stencil():
    p = wl.circle64(32)
    s = gf.assemble_problem(p)
    # node at the centre of the grid is deep inside the disc
    N = p.N
    k = N // 2 + (N // 2) * (N + 1)
    row = s.A[k].toarray().ravel()
    nb = [k + d for d in (-N - 2, -N - 1, -N, -1, 1, N, N + 1, N + 2)]
    assert row[k] == pytest.approx(8.0 / 3.0, abs=1e-14)
    np.testing.assert_allclose(row[nb], -1.0 / 3.0, atol=1e-14)
    assert np.count_nonzero(np.abs(row) > 1e-15) == 9


def _paper_1d(theta, h, lam):
    """Cut-cell block of the 1D system of Sec. 4, Eq. ls1dA / ls1dF
    (cell [x0, x1], x0 ghost, Dirichlet point a with x1 - a = theta h)."""
    AI = theta / h * np.array([[1.0, -1.0], [-1.0, 1.0]])
    AB = np.array([[-theta, theta], [theta - 1.0, 1.0 - theta]]) / h
    Alam = lam * np.array([[theta ** 2, theta * (1 - theta)],
                           [theta * (1 - theta), (1 - theta) ** 2]])
    FB = np.array([-1.0, 1.0]) / h            # times g_a
    Flam = lam * np.array([theta, 1.0 - theta])   # times g_a
    return AI + AB + AB.T + Alam, FB + Flam


@pytest.mark.parametrize("theta", [0.9, 0.5, 0.2, 0.03])
def test_straight_cut_reduces_to_1d_system(theta):
    h = 0.05
    gamma = 2.0
    # internal side is x > a = x0 + (1 - theta) h, psi linear in x
    psi4 = np.array([1.0 - theta, -theta, 1.0 - theta, -theta])
    cc = gf.cut_cell(psi4, 3, 4, -0.5, -0.5, h, gamma)
    assert cc.config == "quad"
    # Sec. 4.4 / Sec. 5.3: C = 1/(theta h) for this quad
    assert cc.C == pytest.approx(1.0 / (theta * h), rel=1e-12)
    A1, F1 = _paper_1d(theta, h, cc.lam)
    # 1D factors in y over [0, h] and the internal-part mass in x
    My = h * np.array([[1 / 3, 1 / 6], [1 / 6, 1 / 3]])
    Sy = np.array([[1.0, -1.0], [-1.0, 1.0]]) / h
    s0 = 1.0 - theta          # internal part s in [s0, 1], s = (x - x0)/h
    i00 = ((1 - s0) ** 3) / 3.0                            # int (1-s)^2
    i01 = (0.5 - 1 / 3) - (s0 ** 2 / 2 - s0 ** 3 / 3)      # int s(1-s)
    i11 = (1 - s0 ** 3) / 3.0                              # int s^2
    Mx = h * np.array([[i00, i01], [i01, i11]])
    # local index a + 2b (a: x-vertex, b: y-vertex)
    Ke_ref = np.kron(My, A1) + np.kron(Sy, Mx)
    np.testing.assert_allclose(cc.Ke, Ke_ref, rtol=1e-12, atol=1e-10 * np.abs(Ke_ref).max())
    # boundary load with g = g_a on every vertex: F1 * int_0^h m_b dy = F1 h/2
    G_ref = np.kron(np.array([h / 2, h / 2]), F1)
    np.testing.assert_allclose(cc.Gk @ np.ones(4), G_ref, rtol=1e-12,
                               atol=1e-12 * np.abs(G_ref).max())


@pytest.mark.parametrize("t1,t2", [(1.0, 1.0), (0.3, 0.7), (0.05, 0.9), (0.01, 0.02),
                                   (0.5, 0.5), (0.9, 0.002)])
def test_c_triangle_equals_eigen_definition(t1, t2):
    h = 0.02
    psi4 = np.array([-1.0, (1 - t1) / t1, (1 - t2) / t2, 3.0])
    cfg, pieces, _ = gf.cut_pieces(psi4)
    ints = gf.cell_integrals(pieces, 0.1, 0.2, h)
    c_def = gf.c_definition(ints.Kn, ints.S)
    assert c_def == pytest.approx(gf.c_triangle(t1, t2, h), rel=1e-10)


@pytest.mark.parametrize("t1,t2", [(1.0, 1.0), (0.3, 0.7), (0.05, 0.9), (0.01, 0.02), (0.9, 0.002)])
def test_c_definition_pieces_equals_c_triangle(t1, t2):
    # cell-local coordinates (origin at the cell corner), as the assembly uses
    h = 0.02
    psi4 = np.array([-1.0, (1 - t1) / t1, (1 - t2) / t2, 3.0])
    cfg, pieces, _ = gf.cut_pieces(psi4)
    assert gf.c_definition_pieces(pieces, 0.0, 0.0, h) == pytest.approx(
        gf.c_triangle(t1, t2, h), rel=1e-13)


@pytest.mark.parametrize("theta", [0.9, 0.3, 0.03, 0.004])
def test_c_definition_pieces_straight_cut(theta):
    # Sec. 5.3 rectangle / Sec. 4.4: C = 1/(theta h) for the straight-cut quad
    h = 0.05
    psi4 = np.array([1.0 - theta, -theta, 1.0 - theta, -theta])
    cfg, pieces, _ = gf.cut_pieces(psi4)
    assert gf.c_definition_pieces(pieces, 0.0, 0.0, h) == pytest.approx(1 / (theta * h), rel=1e-13)


def _c_mp(pieces, dps=40):
    """Brute-force C(K) h in mpmath: exact 3-point Gauss on degree <= 2
    integrands of the monomials x, y, xy (reference cell), 40 digits."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = dps
    r = mp.sqrt(mp.mpf(3) / 5) / 2
    S3 = [mp.mpf(1) / 2 - r, mp.mpf(1) / 2, mp.mpf(1) / 2 + r]
    W3 = [mp.mpf(5) / 18, mp.mpf(8) / 18, mp.mpf(5) / 18]
    g = lambda x, y: [(1, 0), (0, 1), (y, x)]
    M = mp.zeros(3, 3); K = mp.zeros(3, 3)
    for pc in pieces:
        P = [(mp.mpf(a), mp.mpf(b)) for a, b in pc.poly]
        for k in range(1, len(P) - 1):
            A, B, C = P[0], P[k], P[k + 1]
            jac = abs((B[0] - A[0]) * (C[1] - A[1]) - (B[1] - A[1]) * (C[0] - A[0]))
            for s_, ws in zip(S3, W3):
                for t_, wt in zip(S3, W3):
                    x = A[0] + s_ * (1 - t_) * (B[0] - A[0]) + s_ * t_ * (C[0] - A[0])
                    y = A[1] + s_ * (1 - t_) * (B[1] - A[1]) + s_ * t_ * (C[1] - A[1])
                    G = g(x, y)
                    for i in range(3):
                        for j in range(3):
                            M[i, j] += jac * s_ * ws * wt * (G[i][0] * G[j][0] + G[i][1] * G[j][1])
        for pr, qr in pc.segments:
            pa = [mp.mpf(v) for v in pr]; qa = [mp.mpf(v) for v in qr]
            dx, dy = qa[0] - pa[0], qa[1] - pa[1]
            L = mp.sqrt(dx * dx + dy * dy)
            for s_, ws in zip(S3, W3):
                G = g(pa[0] + s_ * dx, pa[1] + s_ * dy)
                dn = [(dy * G[i][0] - dx * G[i][1]) / L for i in range(3)]
                for i in range(3):
                    for j in range(3):
                        K[i, j] += L * ws * dn[i] * dn[j]
    Li = mp.inverse(mp.cholesky(M))
    return float(max(mp.eigsy(Li * K * Li.T)[0]))


def test_c_definition_pieces_high_precision_on_thin_quads():
    # thin and slanted quadrilaterals, and two-triangle saddles: 1e-14
    # against a 40-digit evaluation of the same definition
    rng = np.random.default_rng(7)
    cases = [np.array([-0.02542, -0.033139, 0.97458, 0.966861]),
             np.array([-0.001, -0.3, 0.999, 0.7]),
             np.array([-0.5, 0.9, 0.9, -0.4])]
    for _ in range(6):
        a, b = rng.uniform(1e-3, 0.2, 2)
        cases.append(np.array([-a, -b, 1 - a, 1 - b]))
    for psi4 in cases:
        cfg, pieces, _ = gf.cut_pieces(psi4)
        assert cfg in ("quad", "two_triangles")
        ref = _c_mp(pieces)
        assert gf.c_definition_pieces(pieces, 0.0, 0.0, 1.0) == pytest.approx(ref, rel=1e-14)


def test_c_pentagon_is_triangle_at_one():
    h = 0.1
    assert gf.c_pentagon(h) == pytest.approx(gf.c_triangle(1.0, 1.0, h), rel=1e-15)
    assert gf.c_pentagon(h) == pytest.approx(3 * math.sqrt(2) / h, rel=1e-15)


def test_assigned_C_bounds_definition_for_large_cuts():
    rng = np.random.default_rng(1)
    h = 1.0
    for _ in range(300):
        # pentagon: only v3 external
        psi4 = np.array([-rng.uniform(.01, 1), -rng.uniform(.01, 1),
                         -rng.uniform(.01, 1), rng.uniform(1e-3, 1)])
        cfg, pieces, _ = gf.cut_pieces(psi4)
        ints = gf.cell_integrals(pieces, 0, 0, h)
        assert cfg == "pentagon"
        if ints.length > 0:
            assert gf.c_definition(ints.Kn, ints.S) < gf.c_pentagon(h)
        # hexagon
        psi4 = np.array([-rng.uniform(.5, 1), rng.uniform(1e-3, .4),
                         rng.uniform(1e-3, .4), -rng.uniform(.5, 1)])
        cfg, pieces, _ = gf.cut_pieces(psi4)
        assert cfg == "hexagon"
        ints = gf.cell_integrals(pieces, 0, 0, h)
        assert gf.c_definition(ints.Kn, ints.S) < gf.c_pentagon(h)


def test_element_matrices_h_scaling():
    # in 2D, Ke and Gk are h-independent (lambda ~ 1/h), Mk scales with h^2
    psi4 = np.array([-0.3, 0.4, -0.1, 0.9])
    a = gf.cut_cell(psi4, 0, 0, 0.0, 0.0, 1.0, 2.0)
    b = gf.cut_cell(psi4, 0, 0, 0.0, 0.0, 1e-3, 2.0)
    np.testing.assert_allclose(a.Ke, b.Ke, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(a.Gk, b.Gk, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(a.Mk * 1e-6, b.Mk, rtol=1e-10, atol=1e-20)


def test_local_coercivity_of_cut_cells():
    # lambda = 2 C(K) > C(K): each cut cell's a_K is positive semi-definite
    # with the constants as its only null direction when the segment is
    # non-degenerate
    s = gf.assemble_problem(wl.flower(128))
    for c in s.cut:
        ev = np.linalg.eigvalsh(c.Ke)
        assert ev.min() > -1e-12 * ev.max()
