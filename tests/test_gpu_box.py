"""Strong Dirichlet conditions on the box sides on the GPU (mg_bc.box_sides)
against the oracle, on the rectangle of Sec. 5.3 (the unit square cut by
x = 1 - (1 - theta) h: weak Dirichlet on the cut side, strong on x = 0,
y = 0, y = 1).  Tolerances as test_gpu_parity.py: rows of every level to
1e-13, F (with the box values moved to the right-hand side) to 1e-13,
iterates node-wise, solutions within 1e-10 max|u| (fp64, at the rounding
floor) and 1e-9 (mixed, at 1e-13).  The paper's finding on this domain:
the convergence factor grows with gamma (lambda = gamma / (theta h)); on
the GPU it equals the oracle's to 1e-6.
"""
import numpy as np
import pytest

from oracle import ghostfem as gf
from oracle import multigrid as mg
from paper_2505_05105_gb300 import workloads as wl
from parity_tol import assert_nodewise, assert_solution, node_tolerance, residual

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2505_05105_gb300 import ghostmg
    ghostmg.load()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def solver(p, **kw):
    from paper_2505_05105_gb300 import ghostmg
    return ghostmg.Solver(dev(p.psi), p.N, p.x0, p.y0, p.h, box_sides=True, **kw)


def dof_columns(rows, dof, n):
    """Rows with the entries that couple to nodes that are not DOFs removed
    (the GPU keeps the constant stencil's -1/3 towards a box node, which
    only ever multiplies that node's zero value)."""
    out = rows.copy()
    W = n + 1
    k = np.arange(W * W)
    i, j = k % W, k // W
    for s in range(9):
        di, dj = s % 3 - 1, s // 3 - 1
        ii, jj = i + di, j + dj
        ok = (ii >= 0) & (jj >= 0) & (ii <= n) & (jj <= n)
        q = np.where(ok, ii + jj * W, 0)
        out[~(ok & dof[q]), s] = 0.0
    return out


def oracle_rows(A, n):
    A = A.tocoo()
    out = np.zeros(((n + 1) ** 2, 9))
    di = A.col % (n + 1) - A.row % (n + 1)
    dj = A.col // (n + 1) - A.row // (n + 1)
    np.add.at(out, (A.row, (di + 1) + 3 * (dj + 1)), A.data)
    return out


CASES = [(64, 0.1), (64, 0.5), (128, 0.37), (256, 0.9)]


@pytest.mark.parametrize("N,theta", CASES)
def test_rows_rhs_iterates(N, theta):
    p = wl.rectangle(N, theta)
    s = gf.assemble_problem(p)
    lev = mg.build_hierarchy(s)
    F = s.rhs(p.f, p.g)
    with solver(p) as S:
        assert S.counts()[1] == int(s.dof.sum())
        for l, L in enumerate(lev):
            ref = oracle_rows(L.A, L.n)
            err = np.abs(dof_columns(S.stencil(l), L.dof, L.n) - ref).max() / np.abs(ref).max()
            assert err <= 1e-13, (l, err)
        Fd = torch.zeros(s.n_nodes, dtype=torch.float64, device="cuda")
        S.rhs(dev(p.f), dev(p.g), Fd)
        assert np.abs(host(Fd) - F).max() <= 1e-13 * np.abs(F).max()
        u = torch.zeros(s.n_nodes, dtype=torch.float64, device="cuda")
        u_ref = np.zeros(s.n_nodes)
        for k in range(1, 4):
            u_ref = mg.mg_cycle(lev, 0, u_ref, F, nu1=2, nu2=1, eta=4, order="color4")
            S.cycles(dev(F), u, 1)
            assert_nodewise(host(u), u_ref, node_tolerance(s, F, u_ref, 1e-10, 64 * k), k)


@pytest.mark.parametrize("N,theta", CASES)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solution_parity_box(N, theta, precision):
    p = wl.rectangle(N, theta)
    s = gf.assemble_problem(p)
    F = s.rhs(p.f, p.g)
    ud = gf.direct_solve(s, F)
    tol, floor = (2e-15, 1e-13) if precision == "fp64" else (1e-13, 1e-13)
    with solver(p, precision=precision, max_cycles=300) as S:
        u = torch.zeros(s.n_nodes, dtype=torch.float64, device="cuda")
        info = S.solve(dev(p.f), dev(p.g), u, tol=tol, allow_not_converged=precision == "fp64")
        got = host(u)
    assert info.rel_res <= floor
    assert np.abs(residual(s, F, got)).max() <= 2 * floor * np.abs(F).max()
    assert_solution(got, ud, s, F, 1e-10 if precision == "fp64" else 1e-9, what=(N, theta))
    # second-order discretisation error of the manufactured solution: the
    # oracle's own, at this grid
    inside = (s.psi_s.ravel() < 0) & s.dof
    e = np.abs(got - p.u_exact.ravel())[inside].max()
    e_ref = np.abs(ud - p.u_exact.ravel())[inside].max()
    assert e <= e_ref * (1 + 1e-6) + 1e-12


def test_convergence_factor_grows_with_gamma():
    p = wl.rectangle(128, 0.5)
    rho = []
    for gam in (1.3, 2.0, 5.0, 10.0):
        s = gf.assemble_problem(p, gamma=gam)
        lev = mg.build_hierarchy(s)
        ref, _ = mg.convergence_factor(lev, cycles=20, first=11, order="color4", eta=4)
        with solver(p, gamma=gam) as S:
            Fz = torch.zeros(s.n_nodes, dtype=torch.float64, device="cuda")
            u = dev(s.dof.astype(np.float64))
            rn = [S.residual(Fz, u)[0]]
            for _ in range(20):
                S.cycles(Fz, u, 1)
                rn.append(S.residual(Fz, u)[0])
        got = float(np.mean([rn[m] / rn[m - 1] for m in range(11, 21)]))
        assert got == pytest.approx(ref, rel=1e-6), (gam, got, ref)
        rho.append(got)
    assert all(a < b for a, b in zip(rho, rho[1:])), rho


@pytest.mark.parametrize("theta", [0.37, 0.9])
def test_adjoint_with_box_sides(theta):
    """mg_adjoint on a box handle: dL/df = M^T w and dL/dg = G^T w - B^T w
    (the box values enter F as - B g) against the oracle's dense adjoint,
    1e-9 of each gradient's largest entry; the box nodes carry gradient."""
    p = wl.rectangle(64, theta)
    s = gf.assemble_problem(p)
    rng = np.random.default_rng(61)
    dLdu = rng.standard_normal(s.n_nodes)
    ref_f, ref_g = gf.adjoint(s, dLdu)
    with solver(p, precision="fp64") as S:
        u = torch.zeros(s.n_nodes, dtype=torch.float64, device="cuda")
        S.solve(dev(p.f), dev(p.g), u, tol=1e-13)
        df = torch.zeros_like(u)
        dg = torch.zeros_like(u)
        S.adjoint(dev(dLdu), df, dg)
    ring = np.zeros((p.N + 1, p.N + 1), bool)
    ring[0, :] = ring[-1, :] = ring[:, 0] = ring[:, -1] = True
    assert np.abs(ref_g[ring.ravel()]).max() > 0
    for got, ref in ((host(df), ref_f), (host(dg), ref_g)):
        assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()


def test_box_sides_limits():
    from paper_2505_05105_gb300 import ghostmg as G
    p = wl.rectangle(64, 0.5)
    # without box_sides the same level set reaches the box: rejected
    with pytest.raises(G.GhostMGError) as e:
        G.Solver(dev(p.psi), p.N, p.x0, p.y0, p.h)
    assert e.value.code == G.MG_ERR_INVALID_ARG
