"""Mixed Dirichlet / Neumann boundary conditions on the GPU (MG_BC_MIXED,
mg_solve_bc, mg_rhs_bc) against the oracle.

Problems: the annulus (Dirichlet inner, Neumann outer circle) and the leaf
(Dirichlet x >= 0, Neumann x < 0) of Sec. 5.3 with a manufactured solution,
and a disc cut by a straight Neumann side.  Tolerances as
test_gpu_parity.py: operator rows of every level and cut-cell data to 1e-13
of the largest entry, F = M f + G g_D + N g_N to 1e-13, solutions driven to
the attainable fp64 residual within 1e-10 max|u| + 64 eps S_p of the
oracle's direct solution, mixed precision within 1e-9.  The mixed solves
are driven to 1e-13 (not 1e-12 as in test_gpu_parity.py): with Dirichlet
data on only part of the boundary A is worse conditioned (the annulus at
256^2: a residual of 1e-12 ||F|| still allows errors of ~4e-9 max|u|).
"""
import numpy as np
import pytest

from oracle import ghostfem as gf
from oracle import multigrid as mg
from paper_2505_05105_gb300 import workloads as wl
from parity_tol import assert_nodewise, assert_solution, node_tolerance, residual

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PROBLEMS = {
    "annulus64": lambda: wl.annulus(64),
    "leaf64": lambda: wl.leaf(64),
    "half_disc64": lambda: wl.half_disc(64),
    "annulus256": lambda: wl.annulus(256),
}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2505_05105_gb300 import ghostmg
    ghostmg.load()


@pytest.fixture(scope="module")
def cache():
    return {}


def oracle_for(name, cache):
    if name not in cache:
        p = PROBLEMS[name]()
        s = gf.assemble_problem(p)
        cache[name] = (p, s, mg.build_hierarchy(s))
    return cache[name]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def solver(p, **kw):
    from paper_2505_05105_gb300 import ghostmg
    return ghostmg.Solver(dev(p.psi), p.N, p.x0, p.y0, p.h, neumann_mask=p.neumann_mask, **kw)


def oracle_rows(A, n):
    A = A.tocoo()
    out = np.zeros(((n + 1) ** 2, 9))
    di = A.col % (n + 1) - A.row % (n + 1)
    dj = A.col // (n + 1) - A.row // (n + 1)
    np.add.at(out, (A.row, (di + 1) + 3 * (dj + 1)), A.data)
    return out


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_rows_and_cut_cells(name, cache):
    p, s, lev = oracle_for(name, cache)
    assert any(c.neumann for c in s.cut) and not all(c.neumann for c in s.cut)
    with solver(p) as S:
        for l, L in enumerate(lev):
            ref = oracle_rows(L.A, L.n)
            err = np.abs(S.stencil(l) - ref).max() / np.abs(ref).max()
            assert err <= 1e-13, (l, err)
        cells, data = S.cut_cells()
    assert len(cells) == len(s.cut)
    for t, c in enumerate(s.cut):
        for off, M in ((4, c.Ke), (20, c.Mk), (36, c.Gk)):
            sc = max(np.abs(M).max(), np.abs(c.Ke).max())
            assert np.abs(data[t][off:off + 16] - M.ravel()).max() <= 1e-13 * sc, (t, off)


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_rhs_with_neumann_data(name, cache):
    p, s, lev = oracle_for(name, cache)
    with solver(p) as S:
        for gN in (p.gN, None):
            ref = s.rhs(p.f, p.g, gN)
            F = torch.zeros((p.N + 1) ** 2, dtype=torch.float64, device="cuda")
            S.rhs(dev(p.f), dev(p.g), F, gN=None if gN is None else dev(gN))
            assert np.abs(host(F) - ref).max() <= 1e-13 * np.abs(ref).max()
        # host arrays give the same
        Fh = np.zeros((p.N + 1) ** 2)
        S.rhs(np.ascontiguousarray(p.f.ravel()), np.ascontiguousarray(p.g.ravel()), Fh,
              gN=np.ascontiguousarray(p.gN.ravel()))
        ref = s.rhs(p.f, p.g, p.gN)
        assert np.abs(Fh - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("name", ["annulus64", "leaf64"])
def test_iterate_parity(name, cache):
    p, s, lev = oracle_for(name, cache)
    F = s.rhs(p.f, p.g, p.gN)
    u_ref = np.zeros(s.n_nodes)
    with solver(p) as S:
        u = torch.zeros(s.n_nodes, dtype=torch.float64, device="cuda")
        Fd = dev(F)
        for k in range(1, 4):
            u_ref = mg.mg_cycle(lev, 0, u_ref, F, nu1=2, nu2=1, eta=4, order="color4")
            S.cycles(Fd, u, 1)
            assert_nodewise(host(u), u_ref, node_tolerance(s, F, u_ref, 1e-10, 64 * k),
                            (name, k))


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solution_parity(name, precision, cache):
    p, s, lev = oracle_for(name, cache)
    F = s.rhs(p.f, p.g, p.gN)
    ud = gf.direct_solve(s, F)
    # fp64: driven to its rounding floor (asked for 2e-15, at most 300
    # cycles, accepted at 1e-13); mixed: to 1e-13
    tol, floor = (2e-15, 1e-13) if precision == "fp64" else (1e-13, 1e-13)
    with solver(p, precision=precision, max_cycles=300) as S:
        u = torch.zeros(s.n_nodes, dtype=torch.float64, device="cuda")
        info = S.solve(dev(p.f), dev(p.g), u, tol=tol, gN=dev(p.gN),
                       allow_not_converged=precision == "fp64")
        got = host(u)
    assert info.rel_res <= floor
    assert np.abs(residual(s, F, got)).max() <= 2 * floor * np.abs(F).max()
    assert_solution(got, ud, s, F, 1e-10 if precision == "fp64" else 1e-9, what=name)
    if p.u_exact is not None and name != "half_disc64":
        inside = s.psi_s.ravel() < 0
        # the discretisation error of the manufactured solution (the oracle's
        # own, at this grid), not a parity bar
        e = np.abs(got - p.u_exact.ravel())[inside].max()
        e_ref = np.abs(ud - p.u_exact.ravel())[inside].max()
        assert e <= e_ref * (1 + 1e-6) + 1e-12


def test_bad_neumann_data_rejected():
    """NaN in g_N at a vertex of a Neumann cut cell (where it enters F):
    MG_ERR_INVALID_ARG; away from the Neumann cells g_N is not read."""
    from paper_2505_05105_gb300 import ghostmg as G
    p = wl.annulus(64)
    cls = gf.cell_classes(gf.snap(p.psi, p.h, 1.75))
    jc, ic = np.argwhere((cls == gf.CUT) & (np.asarray(p.neumann_mask) != 0))[0]
    with solver(p) as S:
        u = torch.zeros((p.N + 1) ** 2, dtype=torch.float64, device="cuda")
        gN = p.gN.copy()
        gN[jc, ic] = np.nan
        with pytest.raises(G.GhostMGError) as e:
            S.solve(dev(p.f), dev(p.g), u, gN=dev(gN))
        assert e.value.code == G.MG_ERR_INVALID_ARG
        ref = torch.zeros_like(u)
        S.solve(dev(p.f), dev(p.g), ref, tol=1e-10, gN=dev(p.gN))
        gN = p.gN.copy()
        gN[p.N // 2, p.N // 2] = np.nan        # the annulus' hole: no cell uses it
        S.solve(dev(p.f), dev(p.g), u, tol=1e-10, gN=dev(gN))
        assert torch.equal(u, ref)


def test_neumann_data_ignored_without_neumann_cells():
    """On an all-Dirichlet handle mg_solve_bc equals mg_solve bit for bit."""
    p = wl.circle64(64)
    from paper_2505_05105_gb300 import ghostmg as G
    with G.Solver(dev(p.psi), p.N, p.x0, p.y0, p.h) as S:
        a = torch.zeros((p.N + 1) ** 2, dtype=torch.float64, device="cuda")
        b = torch.zeros_like(a)
        S.solve(dev(p.f), dev(p.g), a, tol=1e-11)
        S.solve(dev(p.f), dev(p.g), b, tol=1e-11, gN=dev(np.ones_like(p.f)))
        assert torch.equal(a, b)


@pytest.mark.parametrize("name", ["annulus64", "leaf64"])
def test_adjoint_with_neumann_data(name, cache):
    """mg_adjoint_bc: dL/df, dL/dg_D and dL/dg_N against the oracle's dense
    adjoint (w = A^{-1} dL/du; M^T w, G^T w, N^T w) at 1e-9 of each
    gradient's largest entry, after a solve to 1e-13."""
    p, s, lev = oracle_for(name, cache)
    rng = np.random.default_rng(41)
    dLdu = rng.standard_normal(s.n_nodes)
    ref_f, ref_g = gf.adjoint(s, dLdu)
    ref_n = gf.adjoint_neumann(s, dLdu)
    with solver(p, precision="fp64") as S:
        u = torch.zeros(s.n_nodes, dtype=torch.float64, device="cuda")
        S.solve(dev(p.f), dev(p.g), u, tol=1e-13, gN=dev(p.gN))
        outs = [torch.zeros(s.n_nodes, dtype=torch.float64, device="cuda") for _ in range(3)]
        S.adjoint(dev(dLdu), outs[0], outs[1], dLdgN=outs[2])
        for got, ref in zip(outs, (ref_f, ref_g, ref_n)):
            got = host(got)
            assert np.all(got[~s.dof] == 0)
            assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()
        # only the Neumann gradient, host arrays
        gn = np.zeros(s.n_nodes)
        S.adjoint(dLdu, None, None, dLdgN=gn)
        assert np.abs(gn - ref_n).max() <= 1e-9 * np.abs(ref_n).max()
