"""Pins for the oracle's assembled system (Eq. disc_bil_form, Eq. disc_rhs).

* Patch test: u in span{1, x, y, xy} (harmonic, in Q1) with f = 0, g = u is
  reproduced exactly by the discrete solution, because Omega_h's boundary is
  the union of the cut segments and the Nitsche form is consistent.  A sign
  error in any Nitsche term, a wrong normal or a wrong quadrature breaks it.
* Symmetric positive definite A (Sec. 4.1) by dense eigenvalues at 8..16 cells.
* Second-order accuracy in max norm on manufactured solutions (Sec. 2).
* Mass and boundary-load sums: sum_ij M_ij = |Omega_h|,
  sum_i (G 1)_i = sum_K lambda_K |Gamma_h cap K|.
"""
import math

import numpy as np
import pytest

from oracle import ghostfem as gf
from paper_2505_05105_gb300 import workloads as wl


@pytest.mark.parametrize("make", [wl.circle64, wl.flower])
def test_patch_test_bilinear_solutions_exact(make):
    p = make(64)
    X, Y = wl.node_grid(p.N, p.x0, p.y0, p.h)
    s = gf.assemble_problem(p)
    for u in (np.ones_like(X), 0.3 + X - 2 * Y, X * Y + 0.5 * X - 0.25):
        F = s.rhs(np.zeros_like(u), u)
        uh = gf.direct_solve(s, F)
        err = np.abs(uh - u.ravel())[s.dof].max()
        assert err < 1e-9, err


@pytest.mark.parametrize("N", [8, 16])
@pytest.mark.parametrize("make", [wl.circle64, wl.flower, wl.paper_hourglass])
def test_spd_dense(N, make):
    s = gf.assemble_problem(make(N))
    d = np.flatnonzero(s.dof)
    A = s.A[d][:, d].toarray()
    assert np.abs(A - A.T).max() < 1e-14 * np.abs(A).max()
    ev = np.linalg.eigvalsh(A)
    assert ev.min() > 0.0


def test_mass_and_load_sums():
    p = wl.flower(64)
    s = gf.assemble_problem(p)
    area = (s.cls == gf.INTERNAL).sum() * p.h ** 2 + sum(c.ints.area for c in s.cut)
    assert s.M.sum() == pytest.approx(area, rel=1e-12)
    lam_len = sum(c.lam * c.ints.length for c in s.cut)
    assert (s.G @ np.ones(s.n_nodes)).sum() == pytest.approx(lam_len, rel=1e-12)


def _max_err(make, N):
    p = make(N)
    s = gf.assemble_problem(p)
    F = s.rhs(p.f, p.g)
    uh = gf.direct_solve(s, F)
    inside = s.psi_s.ravel() < 0
    return np.abs(uh - p.u_exact.ravel())[inside].max()


@pytest.mark.parametrize("make", [wl.circle64, wl.flower])
def test_second_order_convergence(make):
    Ns = (32, 64, 128, 256)
    e = [_max_err(make, N) for N in Ns]
    slope = -np.polyfit(np.log(Ns), np.log(e), 1)[0]
    assert slope > 1.8, (e, slope)


def test_refined_direct_solve_is_exact_to_fp64():
    # residual accumulated in extended precision is at rounding level, and the
    # refined solution agrees with a dense solve to within cond(A) eps
    p = wl.flower(64)
    s = gf.assemble_problem(p)
    F = s.rhs(p.f, p.g)
    u = gf.direct_solve(s, F)
    d = np.flatnonzero(s.dof)
    A = s.A[d][:, d].toarray()
    r = F[d].astype(np.longdouble) - A.astype(np.longdouble) @ u[d].astype(np.longdouble)
    eps = np.finfo(np.float64).eps
    assert float(np.abs(r).max()) <= 8 * eps * float(np.abs(A).sum(1).max() * np.abs(u).max())
    ev = np.linalg.eigvalsh(A)
    kappa = ev[-1] / ev[0]
    ud = np.linalg.solve(A, F[d])
    assert np.abs(ud - u[d]).max() <= 4 * kappa * eps * np.abs(u).max()


def test_rhs_linear_in_data():
    p = wl.flower(32)
    s = gf.assemble_problem(p)
    rng = np.random.default_rng(0)
    f1, f2, g1, g2 = (rng.standard_normal(s.n_nodes) for _ in range(4))
    lhs = s.rhs(2 * f1 - f2, 3 * g1 + g2)
    rhs = 2 * s.rhs(f1, 0 * g1) - s.rhs(f2, 0 * g1) + 3 * s.rhs(0 * f1, g1) + s.rhs(0 * f1, g2)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-14)
