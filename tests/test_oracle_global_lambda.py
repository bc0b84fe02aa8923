"""Pins of the oracle's global stabilisation constant (Sec. 5.2, the global
generalized eigenproblem K v = Lambda M v; ``ghostfem.global_C``).

* A straight vertical cut x = c through the whole box (Omega = {x < c}): the
  FE space is a tensor product, K = Kx (x) My and M = Sx (x) My + Mx (x) Sy,
  so expanding in the eigenvectors of (Sy, My) shows that the largest
  quotient is the 1D one (the y-constant mode).  In 1D with one Dirichlet
  end the global and local problems give C = 1 / (theta_1 h) (Sec. 4.4, the
  numerical test of the global problem in Sec. 4.5), theta_1 h the distance
  from the last internal node to the boundary.
* A vertical strip c1 < x < c2 with two cuts: in 1D the quotient of a
  function that is constant away from the two cut cells, with jumps J_L,
  J_R across them, is (J_L^2 + J_R^2) / (theta_L J_L^2 + theta_R J_R^2) / h,
  so C = 1 / (min(theta_L, theta_R) h).
* Any geometry: the quotient of v sums the cells' K and M parts, and each
  cut cell's part of K is at most C_def(K) times its part of M (the local
  definition, Sec. 5.2), so C_global <= max_K C_def(K).  On the circle the
  global constant is strictly below the largest local one (the cell with
  the largest local constant is helped by its neighbours).
* Neumann cells carry no K: with every cut cell Neumann, C_global = 0.
* The MG convergence factor with lambda = gamma C_global is worse than with
  the local lambda_K = gamma C(K) (the qualitative finding of Sec. 5.2 that
  a uniform penalty hurts MG convergence).
"""
import numpy as np
import pytest

from oracle import ghostfem as gf
from oracle import multigrid as mg
from paper_2505_05105_gb300 import workloads as wl

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def grid(N):
    h = 1.0 / N
    x = -0.5 + h * np.arange(N + 1)
    X, Y = np.meshgrid(x, x)
    return X, Y, h


@pytest.mark.parametrize("N,frac", [(16, 0.9), (16, 0.15), (32, 0.5), (32, 0.3)])
def test_straight_cut_is_one_over_theta_h(N, frac):
    X, Y, h = grid(N)
    c = -0.5 + (N // 2 + frac) * h          # theta = frac from the last internal node
    C = gf.global_C(X - c, N, -0.5, -0.5, h)
    assert abs(C * h - 1.0 / frac) <= 1e-10 / frac


@pytest.mark.parametrize("tl,tr", [(0.3, 0.8), (0.7, 0.25)])
def test_strip_takes_the_smaller_theta(tl, tr):
    N = 16
    X, Y, h = grid(N)
    # left boundary: internal nodes at x >= c1, theta_L h = x_first - c1
    c1 = -0.5 + (4 - tl) * h
    c2 = -0.5 + (11 + tr) * h
    psi = np.maximum(c1 - X, X - c2)
    C = gf.global_C(psi, N, -0.5, -0.5, h)
    assert abs(C * h - 1.0 / min(tl, tr)) <= 1e-10 / min(tl, tr)


def test_below_the_largest_local_constant():
    p = wl.circle64()
    C = gf.global_C(p.psi, p.N, p.x0, p.y0, p.h)
    S = gf.assemble_problem(p)
    c_def = []
    for cc in S.cut:
        _, pieces, _ = gf.cut_pieces(gf.cell_corner_psi(S.psi_s, cc.ic, cc.jc))
        c_def.append(gf.c_definition_pieces(pieces, 0.0, 0.0, p.h))
    assert 0.0 < C <= max(c_def) * (1 + 1e-12)
    assert C < 0.95 * max(c_def)


def test_neumann_cells_carry_no_boundary_term():
    N = 16
    X, Y, h = grid(N)
    psi = X - (-0.5 + 8.4 * h)
    mask = np.ones((N, N), np.uint8)
    assert gf.global_C(psi, N, -0.5, -0.5, h, neumann_mask=mask) == pytest.approx(0.0, abs=1e-9)


def test_global_lambda_enters_every_cut_cell():
    p = wl.circle64()
    C = gf.global_C(p.psi, p.N, p.x0, p.y0, p.h)
    S = gf.assemble_problem(p, c_global=C)
    for cc in S.cut:
        assert cc.lam == 2.0 * C
        Ke = cc.ints.S + cc.lam * cc.ints.Ms - cc.ints.Bn - cc.ints.Bn.T
        assert np.array_equal(cc.Ke, Ke)


def test_global_lambda_slows_multigrid():
    p = wl.circle64()
    C = gf.global_C(p.psi, p.N, p.x0, p.y0, p.h)
    rho = {}
    for name, cg in (("local", None), ("global", C)):
        lv = mg.build_hierarchy(gf.assemble_problem(p, c_global=cg))
        rho[name], _ = mg.convergence_factor(lv, cycles=30, first=21)
    assert rho["local"] <= 0.15
    assert rho["global"] > 2 * rho["local"]
