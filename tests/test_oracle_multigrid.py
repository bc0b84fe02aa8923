"""Pins for the oracle's multigrid components.

* Bilinear transfer: the n = 2 restriction matrix printed in Sec. 5.1
  (tests/golden/restriction_n2.txt).
* Galerkin identity (Sec. 4.3, Sec. 6): the triple product P^T A_h P equals
  the fine bilinear form a_h evaluated directly on the coarse hat functions.
* Gauss-Seidel sweeps against pure-Python node-by-node loops.
* Dense solve = sparse direct solve = converged V-cycle on 8..16 cells.
* Convergence factor of the two-grid scheme with gamma = 2, eta = 4 is about
  0.1, and much worse without the extra cut-cell sweeps (Sec. 5.3).
* The unsmoothed two-grid correction is an A-orthogonal projection
  (Galerkin coarse operator, exact coarse solve); W-cycles and the two-grid
  scheme reach the dense solution, and coincide with the V-cycle on two
  levels.
"""
import os

import numpy as np
import pytest

from oracle import ghostfem as gf
from oracle import multigrid as mg
from paper_2505_05105_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_printed_restriction_n2():
    R_paper = np.loadtxt(os.path.join(GOLDEN, "restriction_n2.txt"))
    P = mg.prolongation(1).toarray()       # coarse n = 1, fine n = 2
    np.testing.assert_array_equal(P.T, R_paper)


def test_prolongation_is_bilinear_interpolation():
    nc = 4
    P = mg.prolongation(nc)
    t = np.linspace(0, 1, nc + 1)
    Xc, Yc = np.meshgrid(t, t)
    tf = np.linspace(0, 1, 2 * nc + 1)
    Xf, Yf = np.meshgrid(tf, tf)
    for fn in (lambda x, y: 1 + 0 * x, lambda x, y: x, lambda x, y: y, lambda x, y: x * y):
        np.testing.assert_allclose(P @ fn(Xc, Yc).ravel(), fn(Xf, Yf).ravel(), atol=1e-15)


def _direct_coarse_operator(system):
    """a_h(Phi_J, Phi_I) with coarse Q1 hats Phi evaluated at the fine cells'
    quadrature points (independent of P and of the triple product)."""
    N, h, x0, y0 = system.N, system.h, system.x0, system.y0
    nc = N // 2
    H = 2 * h
    A = np.zeros(((nc + 1) ** 2, (nc + 1) ** 2))
    cut = {(c.ic, c.jc): c for c in system.cut}
    for jc in range(N):
        for ic in range(N):
            cl = system.cls[jc, ic]
            if cl == gf.EXTERNAL:
                continue
            psi4 = gf.cell_corner_psi(system.psi_s, ic, jc)
            _, pieces, _ = gf.cut_pieces(psi4)
            lam = cut[(ic, jc)].lam if cl == gf.CUT else 0.0
            IC, JC = ic // 2, jc // 2
            Xc, Yc = x0 + IC * H, y0 + JC * H
            nodes = [IC + JC * (nc + 1), IC + 1 + JC * (nc + 1),
                     IC + (JC + 1) * (nc + 1), IC + 1 + (JC + 1) * (nc + 1)]
            loc = np.zeros((4, 4))
            for pc in pieces:
                poly = np.array([[x0 + (ic + a) * h, y0 + (jc + b) * h] for a, b in pc.poly])
                X, W = gf.polygon_rule(poly)
                _, g = gf.q1_shape(X[:, 0], X[:, 1], Xc, Yc, H)
                loc += np.einsum("q,qia,qja->ij", W, g, g)
                for pr, qr in pc.segments:
                    p = np.array([x0 + (ic + pr[0]) * h, y0 + (jc + pr[1]) * h])
                    q = np.array([x0 + (ic + qr[0]) * h, y0 + (jc + qr[1]) * h])
                    d = q - p
                    n = np.array([d[1], -d[0]]) / np.hypot(*d)
                    Xs, Ws = gf.segment_rule(p, q)
                    phi, g = gf.q1_shape(Xs[:, 0], Xs[:, 1], Xc, Yc, H)
                    dn = g @ n
                    loc += lam * np.einsum("q,qi,qj->ij", Ws, phi, phi)
                    loc -= np.einsum("q,qj,qi->ij", Ws, dn, phi)
                    loc -= np.einsum("q,qi,qj->ij", Ws, dn, phi)
            A[np.ix_(nodes, nodes)] += loc
    return A


@pytest.mark.parametrize("make", [wl.circle64, wl.flower])
def test_galerkin_equals_direct_assembly_on_coarse_hats(make):
    s = gf.assemble_problem(make(16))
    lev = mg.build_hierarchy(s, coarsest=8)
    A_tp = lev[1].A.toarray()
    A_dir = _direct_coarse_operator(s)
    np.testing.assert_allclose(A_tp, A_dir, rtol=0, atol=1e-12 * np.abs(A_dir).max())


def test_coarse_dofs_are_vertices_of_active_coarse_cells():
    s = gf.assemble_problem(wl.flower(128))
    lev = mg.build_hierarchy(s)
    for L in lev:
        n = L.n
        m = np.zeros((n + 1, n + 1), dtype=bool)
        jj, ii = np.nonzero(L.cls != gf.EXTERNAL)
        for dj in (0, 1):
            for di in (0, 1):
                m[jj + dj, ii + di] = True
        np.testing.assert_array_equal(m.ravel(), L.dof)
        assert (L.A.diagonal()[L.dof] > 0).all()
        assert (L.A.diagonal()[~L.dof] == 0).all()


def _gs_loop(A, u, F, nodes):
    u = u.copy()
    for p in nodes:
        s = F[p] - A[p] @ u + A[p, p] * u[p]
        u[p] = s / A[p, p]
    return u


@pytest.mark.parametrize("subset", ["all", "cut"])
def test_gs_sweeps_match_node_loops(subset):
    s = gf.assemble_problem(wl.flower(16))
    lev = mg.build_hierarchy(s, coarsest=8)
    L = lev[0]
    A = L.A.toarray()
    rng = np.random.default_rng(3)
    u0 = rng.standard_normal(A.shape[0]) * L.dof
    F = rng.standard_normal(A.shape[0]) * L.dof
    mask = L.dof if subset == "all" else (L.cut_nodes & L.dof)
    # lexicographic in k
    ref = _gs_loop(A, u0, F, np.flatnonzero(mask))
    got = mg.gs_sweep(L, u0.copy(), F, subset, "lex")
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)
    # four colours (0,0), (1,0), (0,1), (1,1)
    n = L.n
    order = [k for c in ((0, 0), (1, 0), (0, 1), (1, 1)) for k in np.flatnonzero(mask)
             if (k % (n + 1)) % 2 == c[0] and (k // (n + 1)) % 2 == c[1]]
    ref = _gs_loop(A, u0, F, order)
    got = mg.gs_sweep(L, u0.copy(), F, subset, "color4")
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("N", [8, 16])
@pytest.mark.parametrize("make", [wl.circle64, wl.flower])
def test_dense_sparse_multigrid_agree(N, make):
    p = make(N)
    s = gf.assemble_problem(p)
    F = s.rhs(p.f, p.g)
    d = np.flatnonzero(s.dof)
    u_dense = np.zeros(s.n_nodes)
    u_dense[d] = np.linalg.solve(s.A[d][:, d].toarray(), F[d])
    u_sp = gf.direct_solve(s, F)
    lev = mg.build_hierarchy(s, coarsest=4)
    u_mg, hist, k = mg.solve(lev, F, tol=1e-14, max_cycles=60)
    scale = np.abs(u_dense).max()
    # cond(A) ~ 1e5 here, so two exact solvers agree to ~cond * eps
    assert np.abs(u_sp - u_dense).max() <= 1e-11 * scale
    assert np.abs(u_mg - u_dense).max() <= 1e-11 * scale
    assert hist[-1] <= 1e-14


@pytest.mark.parametrize("make", [wl.paper_circle, wl.paper_flower, wl.paper_hourglass])
def test_two_grid_convergence_factor(make):
    # Sec. 5.3: local lambda with gamma = 2 and eta = 4 extra cut sweeps gives
    # rho ~ 0.1; without the extra sweeps the factor is far from optimal
    s = gf.assemble_problem(make(64), gamma=2.0, alpha=1.75)
    lev = mg.build_hierarchy(s)
    rho4, _ = mg.convergence_factor(lev, two_grid=True, order="lex", eta=4)
    rho0, _ = mg.convergence_factor(lev, two_grid=True, order="lex", eta=0)
    assert rho4 < 0.15, rho4
    assert rho0 > 0.2 and rho0 > 2.5 * rho4, (rho0, rho4)


def test_vcycle_solves_config1():
    p = wl.circle64(64)
    s = gf.assemble_problem(p)
    lev = mg.build_hierarchy(s)
    F = s.rhs(p.f, p.g)
    u, hist, k = mg.solve(lev, F, tol=1e-10)
    assert hist[-1] <= 1e-10 and k <= 12
    ud = gf.direct_solve(s, F)
    assert np.abs(u - ud).max() <= 1e-9 * np.abs(ud).max()


def test_rediscretised_levels_are_the_coarse_grid_discretisations():
    """Coarse re-discretisation: level l of the 128^2 flower is the ghost-FEM
    system of the same level set on the 2^-l coarser grid (flower(128 / 2^l)
    samples the level set at exactly those nodes)."""
    p = wl.flower(128)
    s = gf.assemble_problem(p)
    lev = mg.build_hierarchy(s, rediscretise_psi=p.psi)
    for l in (1, 2, 3):
        q = wl.flower(128 >> l)
        sq = gf.assemble_problem(q)
        assert lev[l].n == q.N
        assert abs(lev[l].A - sq.A).max() <= 1e-14 * abs(sq.A).max()
        np.testing.assert_array_equal(lev[l].dof, sq.dof)


@pytest.mark.parametrize("make", [wl.paper_circle, wl.paper_flower, wl.paper_hourglass])
def test_rediscretised_cycles_converge(make):
    # the alternative to Eq. galerkin: still a convergent multigrid with the
    # extra cut-cell sweeps (measured rho 0.06-0.11 for V, <= 0.05 for W)
    p = make(64)
    s = gf.assemble_problem(p)
    lev = mg.build_hierarchy(s, rediscretise_psi=p.psi)
    rv, _ = mg.convergence_factor(lev, order="color4", eta=4)
    rw, _ = mg.convergence_factor(lev, order="color4", eta=4, gamma_star=2)
    assert rv < 0.2 and rw < 0.1, (rv, rw)
    F = np.random.default_rng(3).standard_normal(s.n_nodes) * s.dof
    u, hist, k = mg.solve(lev, F, tol=1e-10)
    assert hist[-1] <= 1e-10 and k <= 15


@pytest.mark.parametrize("make", [wl.circle64, wl.flower])
def test_coarse_correction_is_an_a_orthogonal_projection(make):
    """With no smoothing, one two-grid step maps the error e to
    (I - P A_2h^-1 P^T A) e, which for the Galerkin operator A_2h = P^T A P
    (Eq. galerkin) is a projection: applying it twice changes nothing, and
    the corrected error is A-orthogonal to the coarse space (P^T A e = 0).
    A wrong transfer, a non-Galerkin coarse matrix or an inexact coarse solve
    breaks both."""
    p = make(32)
    s = gf.assemble_problem(p)
    lev = mg.build_hierarchy(s)
    rng = np.random.default_rng(3)
    F = np.zeros(s.n_nodes)
    e0 = rng.standard_normal(s.n_nodes) * s.dof
    e1 = mg.mg_cycle(lev, 0, e0.copy(), F, nu1=0, nu2=0, exact_below=1)
    e2 = mg.mg_cycle(lev, 0, e1.copy(), F, nu1=0, nu2=0, exact_below=1)
    scale = np.abs(e1).max()
    assert np.abs(e2 - e1).max() <= 1e-9 * scale
    Ae = lev[0].A @ e1
    assert np.abs(lev[0].P.T @ Ae).max() <= 1e-9 * np.abs(lev[0].A).max() * scale
    assert np.abs(e1 - e0).max() > 1e-3 * np.abs(e0).max()   # it did correct


@pytest.mark.parametrize("make", [wl.circle64, wl.flower])
def test_w_and_two_grid_cycles_reach_the_dense_solution(make):
    """W-cycles (gamma* = 2) and the two-grid scheme (Alg. 1) converge to the
    dense solution, and on a two-level hierarchy (the coarse level is the
    coarsest, solved exactly) V, W and two-grid steps are the same."""
    p = make(16)
    s = gf.assemble_problem(p)
    F = s.rhs(p.f, p.g)
    d = np.flatnonzero(s.dof)
    ud = np.zeros(s.n_nodes)
    ud[d] = np.linalg.solve(s.A[d][:, d].toarray(), F[d])
    scale = np.abs(ud).max()
    lev = mg.build_hierarchy(s, coarsest=4)
    for kw in (dict(gamma_star=2), dict(exact_below=1)):
        u = np.zeros(s.n_nodes)
        for _ in range(40):
            u = mg.mg_cycle(lev, 0, u, F, **kw)
        assert np.abs(u - ud).max() <= 1e-11 * scale, kw
    two = mg.build_hierarchy(s, coarsest=8)
    assert len(two) == 2
    outs = []
    for kw in (dict(gamma_star=1), dict(gamma_star=2), dict(exact_below=1)):
        outs.append(mg.mg_cycle(two, 0, np.zeros(s.n_nodes), F, **kw))
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


@pytest.mark.parametrize("make, nu, eta", [
    (lambda: wl.circle64(16), (2, 1), 4),
    (lambda: wl.flower(32), (2, 1), 4),
    (lambda: wl.flower(32), (1, 2), 2),
])
def test_transposed_cycle_is_the_transpose(make, nu, eta):
    """mg_cycle_transposed is B^T: the approximate inverse of one V-cycle
    from u = 0 (u = B F) and of the transposed cycle, built column by column
    on the DOFs, are transposes of each other; B is not symmetric (V(2,1)
    with a forward Gauss-Seidel), so the test tells them apart."""
    p = make()
    s = gf.assemble_problem(p)
    lev = mg.build_hierarchy(s, coarsest=4)
    d = np.flatnonzero(s.dof)
    B = np.zeros((len(d), len(d)))
    BT = np.zeros_like(B)
    for a, k in enumerate(d):
        e = np.zeros(s.n_nodes)
        e[k] = 1.0
        B[:, a] = mg.mg_cycle(lev, 0, np.zeros(s.n_nodes), e, nu1=nu[0], nu2=nu[1], eta=eta,
                              order="color4")[d]
        BT[:, a] = mg.mg_cycle_transposed(lev, 0, np.zeros(s.n_nodes), e, nu1=nu[0],
                                          nu2=nu[1], eta=eta)[d]
    scale = np.abs(B).max()
    assert np.abs(BT - B.T).max() <= 1e-12 * scale
    assert np.abs(B - B.T).max() > 1e-6 * scale      # ~1e-5: B is not symmetric
