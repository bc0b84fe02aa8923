"""Pins of the oracle's 1D model (Sec. 4; oracle/oned.py).

* The matrix and right-hand side assembled from the element integrals equal
  Eq. ls1dA / Eq. ls1dF entry by entry.
* The proposition of Sec. 4.2: the coarse residual of the splitting strategy
  (Eq. rsplit, with the boundary residuals rebuilt on the coarse grid at
  theta -> (1 + theta) / 2) equals the standard restriction R r_h.
* Sec. 4.3: the Galerkin operator R A_h R^T equals the coarse grid's own
  assembly with theta -> (1 + theta) / 2 and the same lambda.
* Sec. 4.4 / Sec. 4.5: the local 2 x 2 pencil and the global pencil both give
  C = 1 / (theta_1 h).
* Converged two-grid, V- and W-cycles reach the dense solution.
* The qualitative findings of Sec. 4.5: with lambda = 1.1 / (theta_1 h) the
  two-grid scheme and the W-cycle contract by rho ~ 0.1 for every theta_1;
  with lambda = h^-2 the two-grid factor is far from that for most theta_1.
"""
import numpy as np
import pytest

from oracle import oned

CASES = [(16, 0.3, 0.7, 40.0), (32, 0.0099, 0.01, 3500.0), (64, 1.0, 1.0, 64.0),
         (32, 0.75, 0.2, 1.1 * 32 / 0.75)]


@pytest.mark.parametrize("n,t1,t2,lam", CASES)
def test_assembly_matches_the_printed_system(n, t1, t2, lam):
    p = oned.Problem1D(n, t1, t2, lam)
    E = oned.assemble(p)
    P = oned.printed_system(p)
    scale = np.abs(P["A"]).max()
    assert np.abs(E["A"] - P["A"]).max() <= 1e-13 * scale
    assert np.abs(E["gD"] - (P["FB"] + P["Fl"])).max() <= 1e-13 * np.abs(P["Fl"]).max()
    # phi(b) at b = 1 - (1 - theta_2) h: rounding of b, times the slope 1/h
    assert np.abs(E["gN"] - P["FN"]).max() <= 4 * n * np.finfo(float).eps
    # interior rows: 1/h (-1, 2, -1); mass of a whole cell h/6 (2, 1)
    assert np.allclose(E["M"][n // 2, n // 2 - 1:n // 2 + 2], p.h / 6 * np.array([1, 4, 1]),
                       rtol=1e-14, atol=0)


@pytest.mark.parametrize("n,t1,t2,lam", CASES)
def test_splitting_equals_standard_restriction(n, t1, t2, lam):
    p = oned.Problem1D(n, t1, t2, lam)
    rng = np.random.default_rng(n)
    u, f = rng.standard_normal(n + 1), rng.standard_normal(n + 1)
    ga, gb = rng.standard_normal(2)
    E = oned.assemble(p)
    F = E["M"] @ f + E["gD"] * ga + E["gN"] * gb
    r2h = oned.restriction(n) @ (F - E["A"] @ u)
    rs = oned.split_coarse_residual(p, u, f, ga, gb)
    assert np.abs(rs - r2h).max() <= 1e-12 * np.abs(r2h).max()


def test_restriction_is_eq_resop():
    R = oned.restriction(4)
    ref = 0.5 * np.array([[2, 1, 0, 0, 0], [0, 1, 2, 1, 0], [0, 0, 0, 1, 2]], float)
    assert np.array_equal(R, ref)


@pytest.mark.parametrize("n,t1,t2,lam", CASES)
def test_galerkin_equals_coarse_assembly(n, t1, t2, lam):
    p = oned.Problem1D(n, t1, t2, lam)
    R = oned.restriction(n)
    Ac = R @ oned.assemble(p)["A"] @ R.T
    q = oned.Problem1D(n // 2, (1 + t1) / 2, (1 + t2) / 2, lam)
    Ad = oned.assemble(q)["A"]
    assert np.abs(Ac - Ad).max() <= 1e-12 * np.abs(Ad).max()


@pytest.mark.parametrize("n", [128, 1024])
@pytest.mark.parametrize("t1", [0.0099, 0.05, 0.3, 0.75, 1.0])
def test_local_and_global_constant(n, t1):
    p = oned.Problem1D(n, t1, 0.01, 1.0)
    ref = 1.0 / (t1 * p.h)
    assert oned.local_C(p) == pytest.approx(ref, rel=1e-12)
    if n <= 128:
        assert oned.global_C(p) == pytest.approx(ref, rel=1e-9)


@pytest.mark.parametrize("scheme", ["two-grid", "V", "W"])
def test_cycles_reach_the_dense_solution(scheme):
    p = oned.Problem1D(64, 0.3, 0.5, 1.1 / (0.3 / 64))
    E = oned.assemble(p)
    rng = np.random.default_rng(5)
    F = E["M"] @ rng.standard_normal(65) + E["gD"] * 0.7 + E["gN"] * -0.4
    ud = np.linalg.solve(E["A"], F)
    lev = oned.hierarchy(p)
    u = np.zeros(65)
    for _ in range(40):
        u = oned.cycle(lev, 0, u, F, gamma_star=2 if scheme == "W" else 1,
                       two_grid=scheme == "two-grid")
    assert np.abs(u - ud).max() <= 1e-11 * np.abs(ud).max()


def test_convergence_findings_of_sec_4_5():
    n = 256
    h = 1.0 / n
    good, bad, w = [], [], []
    for t1 in (0.0099, 0.05, 0.1, 0.3, 0.5, 0.9, 1.0):
        good.append(oned.convergence_factor(oned.Problem1D(n, t1, 0.01, 1.1 / (t1 * h)))[0])
        bad.append(oned.convergence_factor(oned.Problem1D(n, t1, 0.01, h ** -2))[0])
        w.append(oned.convergence_factor(oned.Problem1D(n, t1, 0.01, 1.1 / (t1 * h)), "W")[0])
    assert max(good) <= 0.1
    assert max(w) <= 0.13
    assert sum(b > 0.5 for b in bad) >= 4
