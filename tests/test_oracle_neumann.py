"""Pins for the oracle's Neumann cut cells (mixed boundary conditions).

* A straight (vertical) Neumann cut reduces to the Neumann end of the 1D
  system printed in Sec. 4: the theta_2 block of Eq. ls1dA (volume term
  only) and F^N of Eq. ls1dF, tensored with 1D Q1 factors in y.  This pins
  the orientation of the Neumann load and the absence of Nitsche terms.
* Patch test: on a disc cut by a straight Neumann side, bilinear harmonic u
  (f = 0, g_D = u on the Dirichlet cells, g_N = du/dx on the straight side)
  is reproduced exactly: a wrong sign or a stray Nitsche term on the Neumann
  cells breaks it.
* Symmetric positive definite A with Neumann cells; the Neumann load sums to
  the length of the Neumann boundary.
* Second-order accuracy in max norm on the annulus (Dirichlet inner, Neumann
  outer circle) and the leaf (Dirichlet x >= 0, Neumann x < 0) of Sec. 5.3.
  The leaf is checked without snapping: snapping (Sec. 2) moves a node onto
  the boundary when it lies within h^alpha of it, which tilts that cell's
  boundary segment by up to h^(alpha - 1), while the Neumann data carry the
  exact normal; with alpha = 1.75 the leaf's max error falls at rate ~1.5 on
  N = 32..256 (it does not with Dirichlet data, which need no normal).
"""
import numpy as np
import pytest

from oracle import ghostfem as gf
from paper_2505_05105_gb300 import workloads as wl


@pytest.mark.parametrize("theta", [0.9, 0.5, 0.2, 0.03])
def test_straight_neumann_cut_reduces_to_1d_end(theta):
    h = 0.05
    # internal side x < b, b at s = theta from the cell's left edge
    psi4 = np.array([-theta, 1.0 - theta, -theta, 1.0 - theta])
    cc = gf.cut_cell(psi4, 3, 4, -0.5, -0.5, h, 2.0, neumann=True)
    assert cc.config == "quad" and cc.neumann
    # Eq. ls1dA: the partial cell contributes theta/h [[1, -1], [-1, 1]]
    A1 = theta / h * np.array([[1.0, -1.0], [-1.0, 1.0]])
    My = h * np.array([[1 / 3, 1 / 6], [1 / 6, 1 / 3]])
    Sy = np.array([[1.0, -1.0], [-1.0, 1.0]]) / h
    i00 = (1 - (1 - theta) ** 3) / 3.0                  # int_0^theta (1-s)^2
    i01 = theta ** 2 / 2 - theta ** 3 / 3               # int_0^theta s(1-s)
    i11 = theta ** 3 / 3.0                              # int_0^theta s^2
    Mx = h * np.array([[i00, i01], [i01, i11]])
    Ke_ref = np.kron(My, A1) + np.kron(Sy, Mx)
    np.testing.assert_allclose(cc.Ke, Ke_ref, rtol=1e-12, atol=1e-10 * np.abs(Ke_ref).max())
    assert np.all(cc.Gk == 0.0)
    # Eq. ls1dF: F^N = (1 - theta, theta) g_b; g = 1 on every vertex,
    # tensored with int_0^h m_b dy = h / 2
    FN = np.array([1.0 - theta, theta])
    np.testing.assert_allclose(cc.Nk @ np.ones(4), np.kron([h / 2, h / 2], FN), rtol=1e-12,
                               atol=1e-15)
    # and with g varying in x only: (Nk g) = F^N (g at b) h/2, g linear
    g = np.array([1.0, 3.0, 1.0, 3.0])                 # g(s) = 1 + 2 s
    np.testing.assert_allclose(cc.Nk @ g, np.kron([h / 2, h / 2], FN * (1 + 2 * theta)),
                               rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("N", [32, 64])
def test_patch_test_straight_neumann_side(N):
    p = wl.half_disc(N)
    assert p.neumann_mask.sum() > 0
    X, Y = wl.node_grid(p.N, p.x0, p.y0, p.h)
    s = gf.assemble_problem(p)
    assert sum(c.neumann for c in s.cut) == int(p.neumann_mask[s.cls == gf.CUT].sum())
    for u, ux in ((np.ones_like(X), np.zeros_like(X)),
                  (0.3 + X - 2 * Y, np.ones_like(X)),
                  (X * Y + 0.5 * X - 0.25, Y + 0.5)):
        F = s.rhs(np.zeros_like(u), u, ux)
        uh = gf.direct_solve(s, F)
        err = np.abs(uh - u.ravel())[s.dof].max()
        assert err < 1e-9, err
    # a wrong sign of the Neumann load is seen
    u, ux = 0.3 + X - 2 * Y, np.ones_like(X)
    uh = gf.direct_solve(s, s.rhs(np.zeros_like(u), u, -ux))
    assert np.abs(uh - u.ravel())[s.dof].max() > 1e-3


@pytest.mark.parametrize("make", [wl.annulus, wl.leaf])
def test_spd_and_neumann_load_sum(make):
    s = gf.assemble_problem(make(16))
    d = np.flatnonzero(s.dof)
    A = s.A[d][:, d].toarray()
    assert np.abs(A - A.T).max() < 1e-14 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0.0
    neu = [c for c in s.cut if c.neumann]
    assert neu and len(neu) < len(s.cut)
    L = sum(c.ints.length for c in neu)
    assert (s.Gn @ np.ones(s.n_nodes)).sum() == pytest.approx(L, rel=1e-12)


def _max_err(make, N, alpha):
    p = make(N)
    s = gf.assemble(p.psi, N, p.x0, p.y0, p.h, 2.0, alpha, p.neumann_mask)
    uh = gf.direct_solve(s, s.rhs(p.f, p.g, p.gN))
    inside = s.psi_s.ravel() < 0
    return np.abs(uh - p.u_exact.ravel())[inside].max()


@pytest.mark.parametrize("make,alpha", [(wl.annulus, 1.75), (wl.leaf, 8.0)])
def test_second_order_convergence_mixed(make, alpha):
    Ns = (32, 64, 128, 256)
    e = [_max_err(make, N, alpha) for N in Ns]
    slope = -np.polyfit(np.log(Ns), np.log(e), 1)[0]
    assert slope > 1.8, (e, slope)
