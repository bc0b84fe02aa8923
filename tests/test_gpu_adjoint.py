"""mg_adjoint and the differentiable solve, on the GPU.

A is symmetric (Sec. 4.1) and F = M f + G g is linear in f and g (Eq.
disc_rhs), so for a loss L(u): w solves A w = dL/du, dL/df = M^T w and
dL/dg = G^T w; mg_adjoint solves for w with the transposed V-cycle (held
to the oracle's transposed cycle iterate by iterate below).  Checked against
  * the oracle's dense adjoint (direct solve, exact to fp64) at small N,
  * central differences of the GPU's own forward solves on the adjoint
    configuration (flower 512^2, loss 1/2 sum over internal nodes of
    (u - u_t)^2, u_t a manufactured solution with seeded phases, 64 sampled
    entries of f and g),
  * torch.autograd through ghostmg.solve_diff.
u is affine in f and g, so central differences carry no truncation error at
any step: the configured step h = 1e-6 is checked at the accuracy its
rounding allows (the loss changes by ~1e-12 there), and a unit step to the
accuracy of the adjoint solve (1e-6 of the gradient's largest entry).
"""
import numpy as np
import pytest

from oracle import ghostfem as gf
from paper_2505_05105_gb300 import workloads as wl

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
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("name,precision", [("circle64", "fp64"), ("flower128", "fp64"),
                                            ("flower128", "mixed")])
def test_adjoint_matches_oracle(name, precision):
    from paper_2505_05105_gb300 import ghostmg as G
    p = wl.circle64(64) if name == "circle64" else wl.flower(128)
    s = gf.assemble_problem(p)
    rng = np.random.default_rng(21)
    dLdu = rng.standard_normal(s.n_nodes)
    ref_f, ref_g = gf.adjoint(s, dLdu)
    S = G.Solver(dev(p.psi), p.N, p.x0, p.y0, p.h, precision=precision)
    # the adjoint solves to the last solve's tolerance (1e-12: above the
    # rounding floor of the unscaled right-hand side dL/du, ~2e-13 here)
    u = torch.zeros(s.n_nodes, dtype=torch.float64, device="cuda")
    S.solve(dev(p.f), dev(p.g), u, tol=1e-12)
    dLdf = torch.zeros_like(u)
    dLdg = torch.zeros_like(u)
    S.adjoint(dev(dLdu), dLdf, dLdg)
    for got, ref in ((host(dLdf), ref_f), (host(dLdg), ref_g)):
        assert np.all(got[~s.dof] == 0)
        assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()
    # one output only; host arrays
    gh = np.zeros(s.n_nodes)
    S.adjoint(dLdu, None, gh)
    assert np.abs(gh - ref_g).max() <= 1e-9 * np.abs(ref_g).max()
    S.close()


@pytest.mark.parametrize("name", ["circle64", "flower128", "discs256", "flower512"])
def test_transposed_cycle_iterates(name):
    """The transposed V-cycle mg_adjoint solves with (mg_cycles_transposed,
    fp64) against the oracle's mg_cycle_transposed, whose operator is pinned
    to be B^T (tests/test_oracle_multigrid.py): iterates after k = 1..3
    cycles node by node, at the fp64 iterate bound of the forward cycle
    (1e-10 max|w| + (64 k eps + ROW_REL) S_p), from w = 0 with a random
    right-hand side on the DOFs (an adjoint dL/du has no smoothness)."""
    from oracle import multigrid as mg
    from paper_2505_05105_gb300 import ghostmg as G
    from parity_tol import assert_nodewise, node_tolerance
    p = {"circle64": lambda: wl.circle64(64), "flower128": lambda: wl.flower(128),
         "discs256": lambda: wl.three_discs(256, seed=0),
         "flower512": lambda: wl.flower(512, k=7, phase=0.3)}[name]()
    s = gf.assemble_problem(p)
    lev = mg.build_hierarchy(s)
    d = np.random.default_rng(8).standard_normal(s.n_nodes) * s.dof
    w_ref = np.zeros(s.n_nodes)
    with G.Solver(dev(p.psi), p.N, p.x0, p.y0, p.h) as S:
        w = torch.zeros(s.n_nodes, dtype=torch.float64, device="cuda")
        dd = dev(d)
        for k in range(1, 4):
            w_ref = mg.mg_cycle_transposed(lev, 0, w_ref, d, nu1=2, nu2=1, eta=4)
            S.cycles_transposed(dd, w, 1)
            torch.cuda.synchronize()
            assert_nodewise(host(w), w_ref, node_tolerance(s, d, w_ref, 1e-10, 64 * k),
                            (name, k))
        # and the bound tells the cycles apart: one forward cycle misses the
        # transposed one by over 100 times the bound (1e3-1e5 measured)
        u = torch.zeros_like(w)
        S.cycles(dd, u, 1)
        w1 = mg.mg_cycle_transposed(lev, 0, np.zeros(s.n_nodes), d, nu1=2, nu2=1, eta=4)
        tol1 = node_tolerance(s, d, w1, 1e-10, 64)
        assert (np.abs(host(u) - w1) / tol1)[s.dof].max() > 100


def test_adjoint_rejects_bad_input():
    from paper_2505_05105_gb300 import ghostmg as G
    p = wl.circle64(64)
    S = G.Solver(dev(p.psi), p.N, p.x0, p.y0, p.h)
    d = np.zeros((p.N + 1) ** 2)
    d[(p.N // 2) * (p.N + 1) + p.N // 2] = np.nan      # a DOF: rejected
    out = torch.zeros((p.N + 1) ** 2, dtype=torch.float64, device="cuda")
    with pytest.raises(G.GhostMGError) as e:
        S.adjoint(dev(d), out, None)
    assert e.value.code == G.MG_ERR_INVALID_ARG
    # dL/du off the DOFs is not read (node (35, 1), outside the disc)
    d = np.zeros((p.N + 1) ** 2)
    d[100] = np.nan
    S.adjoint(dev(d), out, None)
    assert torch.count_nonzero(out) == 0
    with pytest.raises(G.GhostMGError):
        S.adjoint(dev(np.zeros_like(d)), None, None)
    S.close()


def target(p, seed):
    """u_t: the flower's manufactured solution sin 3x cos 2y with seeded phases."""
    return wl.adjoint_target(p, seed)


def test_adjoint_central_differences_flower512():
    """The adjoint configuration: flower 512^2, L = 1/2 sum_internal (u - u_t)^2,
    16 seeded targets; central differences on 64 entries for 4 of them."""
    from paper_2505_05105_gb300 import ghostmg as G
    p = wl.flower(512)
    n = (p.N + 1) ** 2
    S = G.Solver(dev(p.psi), p.N, p.x0, p.y0, p.h, precision="fp64")
    f0, g0 = dev(p.f), dev(p.g)
    inside = dev((np.ravel(p.psi) < 0).astype(float))
    psi_s = gf.snap(p.psi, p.h, 1.75)
    cls = gf.cell_classes(psi_s)
    act = np.zeros((p.N + 1, p.N + 1), bool)
    cut = np.zeros_like(act)
    for dx in (0, 1):
        for dy in (0, 1):
            jj, ii = np.nonzero(cls != gf.EXTERNAL)
            act[jj + dy, ii + dx] = True
            jj, ii = np.nonzero(cls == gf.CUT)
            cut[jj + dy, ii + dx] = True
    rng = np.random.default_rng(22)
    qf = rng.choice(np.flatnonzero(act.ravel()), 32, replace=False)
    qg = rng.choice(np.flatnonzero(cut.ravel()), 32, replace=False)

    def solve(f, g):
        u = torch.zeros(n, dtype=torch.float64, device="cuda")
        S.solve(f, g, u, tol=1e-14, allow_not_converged=True)
        return u

    u0 = solve(f0, g0)
    # the adjoints solve to the last solve's tolerance.  Their right-hand
    # side u - u_t carries no h^2 mass factor, so their fp64 rounding floor
    # relative to ||dL/du|| is ~ eps / h^2 ~ 1e-11: ask for that, accept the
    # floor
    S.solve(f0, g0, torch.zeros(n, dtype=torch.float64, device="cuda"), tol=1e-11)
    targets = [dev(target(p, seed)) for seed in range(16)]
    adjoints = []
    for seed, ut in enumerate(targets):
        dLdu = (u0 - ut) * inside
        dLdf = torch.zeros_like(u0)
        dLdg = torch.zeros_like(u0)
        S.adjoint(dLdu, dLdf, dLdg, allow_not_converged=True)
        assert torch.isfinite(dLdf).all() and torch.isfinite(dLdg).all()
        adjoints.append((host(dLdf), host(dLdg)))
    # the perturbed solves do not depend on the target: reuse them for 4 seeds
    # at h = 1e-6 the two solutions differ by ~1e-11 while each carries
    # rounding of ~1e-14 (times the solve's condition), so the difference is
    # good to ~1e-2 of the gradient's scale; at h = 1 to the adjoint's 1e-6
    for step, tol in ((1e-6, 1e-2), (1.0, 1e-6)):
        for which, qs in (("f", qf), ("g", qg)):
            for q in qs:
                e = torch.zeros(n, dtype=torch.float64, device="cuda")
                e[int(q)] = step
                if which == "f":
                    up, um = solve(f0 + e, g0), solve(f0 - e, g0)
                else:
                    up, um = solve(f0, g0 + e), solve(f0, g0 - e)
                for seed in range(4):
                    ut = targets[seed]
                    adj = adjoints[seed][0 if which == "f" else 1]
                    scale = np.abs(adj).max()
                    # L(u+) - L(u-) = 1/2 sum (u+ - u-) (u+ + u- - 2 u_t) over
                    # internal nodes, evaluated without cancelling L's
                    fd = float((0.5 * (up - um) * (up + um - 2 * ut) * inside).sum()) / (2 * step)
                    assert abs(fd - adj[q]) <= tol * scale, (seed, which, int(q), step, fd, adj[q])
    S.close()


def test_solve_diff_autograd():
    from paper_2505_05105_gb300 import ghostmg as G
    p = wl.flower(128)
    s = gf.assemble_problem(p)
    S = G.Solver(dev(p.psi), p.N, p.x0, p.y0, p.h, precision="fp64")
    f = dev(p.f).requires_grad_(True)
    g = dev(p.g).requires_grad_(True)
    ut = dev(target(p, 5))
    inside = dev((np.ravel(p.psi) < 0).astype(float))
    u = G.solve_diff(S, f, g, tol=1e-13)
    L = 0.5 * ((u - ut) ** 2 * inside).sum()
    L.backward()
    ref_f, ref_g = gf.adjoint(s, host((u - ut) * inside))
    assert np.abs(host(f.grad) - ref_f).max() <= 1e-9 * np.abs(ref_f).max()
    assert np.abs(host(g.grad) - ref_g).max() <= 1e-9 * np.abs(ref_g).max()
    # directional derivative along a random direction (u affine: unit step)
    rng = np.random.default_rng(23)
    v = dev(rng.standard_normal(s.n_nodes))
    with torch.no_grad():
        def Lof(ff):
            uu = torch.zeros_like(ff)
            S.solve(ff, g.detach(), uu, tol=1e-14, allow_not_converged=True)
            return uu
        up, um = Lof(f.detach() + v), Lof(f.detach() - v)
        fd = float((0.5 * (up - um) * (up + um - 2 * ut) * inside).sum()) / 2.0
    assert fd == pytest.approx(float((f.grad * v).sum()), rel=1e-8)
    # only g requires grad: f gets none
    f2 = dev(p.f)
    g2 = dev(p.g).requires_grad_(True)
    u2 = G.solve_diff(S, f2, g2, tol=1e-13)
    (0.5 * ((u2 - ut) ** 2 * inside).sum()).backward()
    assert f2.grad is None and g2.grad is not None
    S.close()
