"""The 1D model of Sec. 4 on the GPU (mg1d_cycles) against the oracle
(oracle/oned.py).

* Residual histories ||F - A u^(m)||_inf, m = 0..50, of the homogeneous
  problem from u = 1 (Sec. 4.5) for the two-grid scheme with lambda = h^-2
  and with lambda = 1.1 / (theta_1 h) (h = 2^-7, 2^-10), and for V- and
  W-cycles with the latter (h = 2^-7, 2^-9), over theta_1 from the paper's
  list, each set in one call.  The histories fall by up to 1e-70, and after
  some cycles they are set by slowly decaying modes that rounding injects
  (the vector of ones holds little of them): a perturbation of u^(0) by
  1e-14 changes the late residuals by O(1) and rho by up to ~15%.  So each
  entry is compared within 1e-9 relative of the oracle's over the prefix
  the arithmetic fixes (at least 8 cycles), and rho over cycles 41..50
  within the spread such a perturbation causes (at least 25%).
* The convergence factors of Sec. 4.5 from those histories: rho <= 0.1 for
  the two-grid scheme with lambda = 1.1 / (theta_1 h), far from it with
  lambda = h^-2.
* A non-homogeneous problem: after 5 V-cycles from 0 the iterate equals the
  oracle's (1e-10 of max|u|), after 20 more the dense solution.
* Invalid arguments are refused.
"""
import numpy as np
import pytest

from oracle import oned

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

THETAS = (0.0099, 0.05, 0.1, 0.3, 0.5, 0.75, 0.9, 1.0)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2505_05105_gb300 import ghostmg
    ghostmg.load()


def run(probs, cycle, cycles=50, F=None, u0=None):
    from paper_2505_05105_gb300 import ghostmg as G
    total = sum(n + 1 for n, *_ in probs)
    u = torch.ones(total, dtype=torch.float64, device="cuda") if u0 is None else u0
    res = G.mg1d_cycles(probs, u, F=F, cycle=cycle, cycles=cycles)
    torch.cuda.synchronize()
    return res, u


def trusted_prefix(p, scheme, rn):
    """Cycles whose residual the arithmetic fixes: the oracle's history from
    u = 1 + 1e-14 noise (a perturbation of the size rounding makes) agrees
    with the one from u = 1 to 1e-9 there.  Later the history is set by
    modes that rounding injects and that decay more slowly than those of
    u = 1, so it differs between any two fp64 implementations."""
    rng = np.random.default_rng(p.n)
    u0 = 1.0 + 1e-14 * rng.standard_normal(p.n + 1)
    rho_p, rp = oned.convergence_factor(p, scheme, u0=u0)
    ok = np.abs(np.array(rp) - rn) <= 1e-9 * rn
    k = int(np.argmin(ok)) if not ok.all() else len(rn)
    return k, rho_p


@pytest.mark.parametrize("scheme,lam_kind", [("two-grid", "h^-2"), ("two-grid", "opt"),
                                             ("V", "opt"), ("W", "opt")])
def test_residual_histories(scheme, lam_kind):
    probs = []
    for m in ((7, 10) if scheme == "two-grid" else (7, 9)):
        n = 2 ** m
        h = 1.0 / n
        for t1 in THETAS:
            probs.append((n, t1, 0.01, h ** -2 if lam_kind == "h^-2" else 1.1 / (t1 * h)))
    res, _ = run(probs, scheme)
    rhos = []
    for k, (n, t1, t2, lam) in enumerate(probs):
        p = oned.Problem1D(n, t1, t2, lam)
        rho, rn = oned.convergence_factor(p, scheme)
        rn = np.array(rn)
        kt, rho_p = trusted_prefix(p, scheme, rn)
        assert kt >= 8, (n, t1, kt)
        assert np.all(np.abs(res[k][:kt] - rn[:kt]) <= 1e-9 * rn[:kt]), (n, t1, scheme)
        got = float(np.mean(res[k][41:51] / res[k][40:50]))
        # past the trusted prefix: within the spread that a rounding-size
        # change of u^(0) causes (measured above), at least 25%
        assert abs(got - rho) <= max(3 * abs(rho_p - rho), 0.25 * rho), (n, t1, got, rho)
        rhos.append(got)
    if scheme == "two-grid" and lam_kind == "opt":
        assert max(rhos) <= 0.1
    if lam_kind == "h^-2":
        assert sum(r > 0.5 for r in rhos) >= 6
    print(scheme, lam_kind, " ".join(f"{r:.3f}" for r in rhos))


def test_nonhomogeneous_solve():
    n, t1, t2 = 512, 0.3, 0.6
    p = oned.Problem1D(n, t1, t2, 1.1 / (t1 / n))
    E = oned.assemble(p)
    x = np.linspace(0.0, 1.0, n + 1)
    F = E["M"] @ (np.pi ** 2 * np.sin(np.pi * x)) + E["gD"] * 0.25 + E["gN"] * -1.5
    ud = np.linalg.solve(E["A"], F)
    scale = np.abs(ud).max()
    lev = oned.hierarchy(p)
    u_ref = np.zeros(n + 1)
    for _ in range(5):
        u_ref = oned.cycle(lev, 0, u_ref, F)
    Fd = torch.from_numpy(F).cuda()
    u = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
    # 5 cycles: still 1e-5 away from the solution, the iterates agree to
    # rounding (cond(A) ~ 5e5 times eps)
    _, u = run([(n, t1, t2, p.lam)], "V", cycles=5, F=Fd, u0=u)
    assert np.abs(u.cpu().numpy() - u_ref).max() <= 1e-10 * scale
    res, u = run([(n, t1, t2, p.lam)], "V", cycles=20, F=Fd, u0=u)
    assert np.abs(u.cpu().numpy() - ud).max() <= 1e-10 * scale
    assert res[0][-1] <= 1e-12 * np.abs(F).max()


def test_refused_arguments():
    from paper_2505_05105_gb300 import ghostmg as G
    u = torch.ones(4097, dtype=torch.float64, device="cuda")
    for bad in ([(1000, 0.5, 0.5, 10.0)], [(8, 0.5, 0.5, 10.0)], [(4096, 0.5, 0.5, 10.0)],
                [(1024, 0.0, 0.5, 10.0)], [(1024, 0.5, 1.5, 10.0)],
                [(1024, 0.5, 0.5, -1.0)], [(1024, 0.5, 0.5, float("nan"))]):
        with pytest.raises(G.GhostMGError) as e:
            G.mg1d_cycles(bad, u)
        assert e.value.code == G.MG_ERR_INVALID_ARG
    with pytest.raises(G.GhostMGError) as e:
        G.mg1d_cycles([(1024, 0.5, 0.5, 10.0)], u.cpu())
    assert e.value.code == G.MG_ERR_INVALID_ARG
