"""GPU edge cases: invalid inputs, degenerate domains and non-default
parameters (eta, nu1, nu2, coarsest level), each against the oracle."""
import numpy as np
import pytest

from oracle import ghostfem as gf
from oracle import multigrid as mg
from paper_2505_05105_gb300 import workloads as wl
from parity_tol import assert_nodewise, assert_solution, node_tolerance

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


def setup_status(psi, N, x0=-0.5, y0=-0.5, h=None, coarsest=8, bc=None, **stab_kw):
    from paper_2505_05105_gb300 import ghostmg as G
    h = 1.0 / N if h is None else h
    stab = G.mg_default_stab()
    for k, v in stab_kw.items():
        setattr(stab, k, v)
    out = G.ctypes.c_void_p()
    lib = G.load()
    psi_d = dev(psi)
    rc = lib.mg_setup(G.ctypes.byref(out), psi_d.data_ptr(),
                      G.ctypes.byref(G.mg_grid(N, x0, y0, h, coarsest)),
                      G.ctypes.byref(bc) if bc is not None else None,
                      G.ctypes.byref(stab), None)
    if out.value:
        lib.mg_destroy(out.value)
    return rc


def test_invalid_setups():
    from paper_2505_05105_gb300 import ghostmg as G
    p = wl.circle64(64)
    assert setup_status(p.psi, 64) == G.MG_OK
    bad = p.psi.copy(); bad[10, 10] = np.nan
    assert setup_status(bad, 64) == G.MG_ERR_INVALID_ARG
    edge = p.psi.copy(); edge[0, 5] = -1.0           # Omega touches the outer ring
    assert setup_status(edge, 64) == G.MG_ERR_INVALID_ARG
    q = wl.circle64(48)
    assert setup_status(q.psi, 48) == G.MG_ERR_INVALID_ARG     # not a power of two
    assert setup_status(p.psi, 64, coarsest=3) == G.MG_ERR_INVALID_ARG
    assert setup_status(p.psi, 64, coarsest=128) == G.MG_ERR_INVALID_ARG
    assert setup_status(p.psi, 64, eta=9) == G.MG_ERR_INVALID_ARG
    mask = (G.ctypes.c_uint8 * (64 * 64))()
    # a mask needs kind MG_BC_MIXED, MG_BC_MIXED needs a mask, unknown kinds
    bc = G.mg_bc(G.MG_BC_DIRICHLET, G.ctypes.cast(mask, G.ctypes.c_void_p))
    assert setup_status(p.psi, 64, bc=bc) == G.MG_ERR_INVALID_ARG
    assert setup_status(p.psi, 64, bc=G.mg_bc(G.MG_BC_MIXED, None)) == G.MG_ERR_INVALID_ARG
    assert setup_status(p.psi, 64, bc=G.mg_bc(5, None)) == G.MG_ERR_INVALID_ARG
    bc = G.mg_bc(G.MG_BC_MIXED, G.ctypes.cast(mask, G.ctypes.c_void_p))
    assert setup_status(p.psi, 64, bc=bc) == G.MG_OK           # all-zero mask
    assert setup_status(p.psi, 64, precision=7) == G.MG_ERR_INVALID_ARG


def test_nan_in_data_rejected():
    """NaN/Inf where the data enter F (f at a vertex of an active cell, g at
    a vertex of a cut cell) or in a DOF entry of u: MG_ERR_INVALID_ARG, the
    handle stays usable.  Entries that never enter the computation (f and u
    outside the domain's cells) are not read: the solve is unchanged."""
    from paper_2505_05105_gb300 import ghostmg as G
    from oracle import ghostfem as gf
    p = wl.circle64(64)
    cls = gf.cell_classes(gf.snap(p.psi, p.h, 1.75))
    jc, ic = np.argwhere(cls == gf.CUT)[0]
    S = G.Solver(dev(p.psi), p.N, p.x0, p.y0, p.h)
    m = (p.N + 1) ** 2
    u = torch.zeros(m, dtype=torch.float64, device="cuda")
    ref = torch.zeros_like(u)
    S.solve(dev(p.f), dev(p.g), ref, tol=1e-10)
    bad_f = p.f.copy(); bad_f[p.N // 2, p.N // 2] = np.inf
    bad_g = p.g.copy(); bad_g[jc, ic] = np.nan
    for f, g in ((bad_f, p.g), (p.f, bad_g)):
        with pytest.raises(G.GhostMGError) as e:
            S.solve(dev(f), dev(g), u)
        assert e.value.code == G.MG_ERR_INVALID_ARG
        with pytest.raises(G.GhostMGError) as e:
            S.rhs(dev(f), dev(g), torch.zeros_like(u))
        assert e.value.code == G.MG_ERR_INVALID_ARG
    u_bad = torch.zeros_like(u)
    u_bad[(p.N // 2) * (p.N + 1) + p.N // 2] = float("nan")
    with pytest.raises(G.GhostMGError) as e:
        S.solve(dev(p.f), dev(p.g), u_bad)
    assert e.value.code == G.MG_ERR_INVALID_ARG
    # outside every active cell: ignored
    far_f = p.f.copy(); far_f[3, 4] = np.inf
    u_far = torch.zeros_like(u)
    u_far[3 * (p.N + 1) + 4] = float("nan")
    info = S.solve(dev(far_f), dev(p.g), u_far, tol=1e-10)
    assert info.rel_res <= 1e-10 and torch.equal(u_far, ref)
    # the handle stays usable
    info = S.solve(dev(p.f), dev(p.g), u, tol=1e-10)
    assert info.rel_res <= 1e-10
    S.close()


def test_empty_domain():
    from paper_2505_05105_gb300 import ghostmg as G
    N = 32
    psi = np.ones((N + 1, N + 1))
    S = G.Solver(dev(psi), N, -0.5, -0.5, 1.0 / N)
    assert S.counts()[1] == 0
    u = torch.ones((N + 1) ** 2, dtype=torch.float64, device="cuda")
    z = torch.zeros_like(u)
    info = S.solve(z, z, u)
    assert info.cycles == 0 and torch.count_nonzero(u) == 0
    S.close()


def test_not_converged_reported():
    from paper_2505_05105_gb300 import ghostmg as G
    p = wl.flower(128)
    S = G.Solver(dev(p.psi), p.N, p.x0, p.y0, p.h, max_cycles=1)
    u = torch.zeros((p.N + 1) ** 2, dtype=torch.float64, device="cuda")
    info = S.solve(dev(p.f), dev(p.g), u, tol=1e-14, allow_not_converged=True)
    assert info.cycles == 1 and info.rel_res > 1e-14
    with pytest.raises(G.GhostMGError) as e:
        S.solve(dev(p.f), dev(p.g), u, tol=1e-14)
    assert e.value.code == G.MG_ERR_NOT_CONVERGED
    S.close()


@pytest.mark.parametrize("eta,nu1,nu2,coarsest", [(0, 2, 1, 8), (1, 1, 1, 4), (3, 1, 2, 16),
                                                   (4, 3, 0, 2), (8, 2, 1, 8)])
def test_parameters_iterate_parity(eta, nu1, nu2, coarsest):
    from paper_2505_05105_gb300 import ghostmg as G
    # 256^2: the fine level, fused intermediate levels (128), the tail block
    p = wl.flower(256, k=3, phase=0.4)
    s = gf.assemble_problem(p)
    lev = mg.build_hierarchy(s, coarsest=coarsest)
    F = s.rhs(p.f, p.g)
    u_ref = np.zeros(s.n_nodes)
    for _ in range(3):
        u_ref = mg.mg_cycle(lev, 0, u_ref, F, nu1=nu1, nu2=nu2, eta=eta, order="color4")
    S = G.Solver(dev(p.psi), p.N, p.x0, p.y0, p.h, eta=eta, nu1=nu1, nu2=nu2,
                 coarsest=coarsest)
    u = torch.zeros(s.n_nodes, dtype=torch.float64, device="cuda")
    S.cycles(dev(F), u, 3)
    torch.cuda.synchronize()
    got = u.cpu().numpy()
    S.close()
    assert_nodewise(got, u_ref, node_tolerance(s, F, u_ref, 1e-10, 64 * 3))


def test_tiny_domain_and_saddle_cells():
    # a disc of radius 2.3 h: a handful of DOFs, every cell cut; and a level
    # set with saddle (diagonal) cut cells
    from paper_2505_05105_gb300 import ghostmg as G
    N = 32
    X, Y = wl.node_grid(N, -0.5, -0.5, 1.0 / N)
    for psi in (np.hypot(X - 0.013, Y + 0.021) - 2.3 / N,
                np.minimum(np.hypot(X - 0.11, Y - 0.1) - 0.2, np.hypot(X + 0.11, Y + 0.12) - 0.2)):
        p = wl.Problem("t", N, -0.5, -0.5, 1.0 / N, psi, np.sin(X), np.cos(Y))
        s = gf.assemble_problem(p)
        ud = gf.direct_solve(s, s.rhs(p.f, p.g))
        S = G.Solver(dev(psi), N, -0.5, -0.5, 1.0 / N)
        u = torch.zeros(s.n_nodes, dtype=torch.float64, device="cuda")
        S.solve(dev(p.f), dev(p.g), u, tol=1e-13)
        torch.cuda.synchronize()
        F = s.rhs(p.f, p.g)
        assert_solution(u.cpu().numpy(), ud, s, F, 1e-10)
        S.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_check_schedule(precision):
    """Residual checks after groups of V-cycles: the adaptive schedule reaches
    the same tolerance as checking after every cycle, with at most one extra
    cycle and fewer fp64 residual evaluations."""
    from paper_2505_05105_gb300 import ghostmg as G
    p = wl.flower(256)
    out = {}
    for inner in (1, 0, 5):
        S = G.Solver(dev(p.psi), p.N, p.x0, p.y0, p.h, precision=precision, inner=inner)
        u = torch.zeros((p.N + 1) ** 2, dtype=torch.float64, device="cuda")
        info = S.solve(dev(p.f), dev(p.g), u, tol=1e-10)
        assert info.rel_res <= 1e-10
        hist = info.history()
        assert len(hist) == info.checks + 1 and hist[-1] == pytest.approx(info.rel_res)
        out[inner] = (info.cycles, info.checks)
        S.close()
    every = out[1]
    assert every[1] == every[0]                       # one check per cycle
    assert out[0][0] <= every[0] + 1 and out[0][1] < every[1]
    assert out[5][0] % 5 == 0 and out[5][1] == out[5][0] // 5


def test_handles_with_different_shared_memory_needs_coexist():
    """Handles whose kernels need different amounts of shared memory (the
    single-block tail's layout depends on the geometry, the fused step's on
    eta) and a batch are alive at once and solve in any order."""
    from paper_2505_05105_gb300 import ghostmg as G
    probs = [(wl.flower(1024, k=7, phase=0.3), dict(eta=8)),
             (wl.circle64(64), dict(eta=2)),
             (wl.three_discs(512, seed=1), dict(eta=4))]
    solvers = [G.Solver(dev(p.psi), p.N, p.x0, p.y0, p.h, precision="mixed", **kw)
               for p, kw in probs]
    B = G.BatchSolver([wl.batch_geometry(i, seed=3) for i in range(4)])
    for rnd in range(2):
        for (p, _), S in zip(probs, solvers):
            u = torch.zeros((p.N + 1) ** 2, dtype=torch.float64, device="cuda")
            assert S.solve(dev(p.f), dev(p.g), u, tol=1e-10).rel_res <= 1e-10
        if rnd == 0:
            # a new handle in between (its setup configures the kernels again)
            solvers.append(G.Solver(dev(wl.flower(128).psi), 128, -0.5, -0.5, 1 / 128,
                                    precision="mixed", eta=1))
    for x in solvers:
        x.close()
    B.close()
