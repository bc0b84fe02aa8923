"""Pins for strong Dirichlet conditions on the box sides (the rectangle of
Sec. 5.3: weak Nitsche Dirichlet on the cut side x = 1 - (1 - theta) h,
strong Dirichlet on x = 0, y = 0, y = 1).

* Patch test: bilinear harmonic u (f = 0, g = u at every node) is
  reproduced exactly: the strong values enter through the couplings moved to
  the right-hand side, the weak side through the Nitsche terms.
* Second-order accuracy in max norm (N = 32..256).
* A is symmetric positive definite on the DOFs, which exclude the box nodes.
* The multigrid hierarchy keeps the coarse box nodes out of the DOFs and the
  V-cycle solves to 1e-10.
"""
import numpy as np
import pytest

from oracle import ghostfem as gf
from oracle import multigrid as mg
from paper_2505_05105_gb300 import workloads as wl


@pytest.mark.parametrize("theta", [0.1, 0.37, 0.9])
def test_patch_test_box(theta):
    p = wl.rectangle(32, theta)
    s = gf.assemble_problem(p)
    X, Y = wl.node_grid(p.N, p.x0, p.y0, p.h)
    ring = np.zeros((p.N + 1, p.N + 1), bool)
    ring[0, :] = ring[-1, :] = ring[:, 0] = ring[:, -1] = True
    assert not np.any(s.dof & ring.ravel())
    for u in (np.ones_like(X), 0.3 + X - 2 * Y, X * Y + 0.5 * X - 0.25):
        uh = gf.direct_solve(s, s.rhs(np.zeros_like(u), u))
        assert np.abs(uh - u.ravel())[s.dof].max() < 1e-11


def test_second_order_convergence_box():
    Ns = (32, 64, 128, 256)
    e = []
    for N in Ns:
        p = wl.rectangle(N, 0.37)
        s = gf.assemble_problem(p)
        uh = gf.direct_solve(s, s.rhs(p.f, p.g))
        inside = (s.psi_s.ravel() < 0) & s.dof
        e.append(np.abs(uh - p.u_exact.ravel())[inside].max())
    slope = -np.polyfit(np.log(Ns), np.log(e), 1)[0]
    assert slope > 1.9, (e, slope)


def test_spd_and_hierarchy_box():
    p = wl.rectangle(16, 0.5)
    s = gf.assemble_problem(p)
    d = np.flatnonzero(s.dof)
    A = s.A[d][:, d].toarray()
    assert np.abs(A - A.T).max() < 1e-14 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0.0
    p = wl.rectangle(64, 0.5)
    s = gf.assemble_problem(p)
    lev = mg.build_hierarchy(s)
    for L in lev:
        jn, in_ = np.divmod(np.arange((L.n + 1) ** 2), L.n + 1)
        ring = (in_ == 0) | (jn == 0) | (in_ == L.n) | (jn == L.n)
        assert not np.any(L.dof & ring)
    F = s.rhs(p.f, p.g)
    u, hist, k = mg.solve(lev, F, tol=1e-10)
    assert hist[-1] <= 1e-10 and k <= 15
    ud = gf.direct_solve(s, F)
    assert np.abs(u - ud).max() <= 1e-8 * np.abs(ud).max()
