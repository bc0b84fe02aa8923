"""GPU parity of the fp32 V-cycle kernels -- the ones the mixed-precision
solve runs and the benchmark times -- against the oracle's fp64 4-colour
V(2,1)-cycle, iterate by iterate.

One refinement step (mg_cycles with MG_MIXED) from an fp64 iterate u0 computes
r = F - A u0 in fp64, scales it by a power of two, runs `inner` fp32 V-cycles
on A e = sigma r from e = 0 and adds e / sigma to u0 in fp64.  V-cycles are
affine in the iterate (Sec. 3.2: u <- u + B (F - A u) with B linear), so in
exact arithmetic the step equals `inner` fp64 V-cycles of the oracle from u0
(oracle.multigrid.mg_cycle, Sec. 4.1 smoother, Sec. 5.1 transfers, Sec. 5.3
extra cut-cell sweeps).  The two differ by the fp32 rounding of the
correction, bounded node-wise by tests/parity_tol.fp32_step_tolerance:
C32 inner 2^-24 (max|e| + S_p(e)) + 64 eps S_p(u).  A wrong restriction
weight, a missing or misplaced extra sweep or a wrong colour order in any
fp32 kernel changes the step by far more (the cycle contracts the error by
~0.1-0.3 per cycle; such a change alters e at O(1) relative).

Kernels covered: the fine fp32 sweep in its three load modes (e = 0 start,
plain, prolongation added on load), the fp32 extra-sweep kernel, the fp32
residual + restriction, the fused smoothing steps of the intermediate levels
(default) or -- with fuse_max_tiles = -1 -- the separate fp32 sweep, extra
sweep and restriction kernels on every level above the tail, the tail block
(levels <= 64 x 64 cells, fp64 coarsest solve), the fp64 refinement
residual and update.
"""
import numpy as np
import pytest

from oracle import ghostfem as gf
from oracle import multigrid as mg
from paper_2505_05105_gb300 import workloads as wl
from parity_tol import assert_nodewise, fp32_step_tolerance

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


PROBLEMS = {
    "circle64": lambda: wl.circle64(64),
    "flower128": lambda: wl.flower(128),
    "discs256": lambda: wl.three_discs(256, seed=0),
    "flower512": lambda: wl.flower(512, k=7, phase=0.3),
}


@pytest.fixture(scope="module")
def oracle_cache():
    return {}


def oracle_for(name, cache):
    if name not in cache:
        p = PROBLEMS[name]()
        s = gf.assemble_problem(p)
        lev = mg.build_hierarchy(s)
        F = s.rhs(p.f, p.g)
        if not np.abs(F).max() > 0:
            F = np.random.default_rng(11).standard_normal(s.n_nodes) * s.dof
        cache[name] = (p, s, lev, F)
    return cache[name]


def starts(s, lev, F, eta):
    """Iterates to start a step from: zero; one fp64 V-cycle from zero
    (smooth error); the latter plus seeded noise on the DOFs (rough error)."""
    u1 = mg.mg_cycle(lev, 0, np.zeros(s.n_nodes), F, nu1=2, nu2=1, eta=eta, order="color4")
    noise = np.random.default_rng(3).standard_normal(s.n_nodes) * s.dof
    rough = u1 + 1e-2 * np.abs(u1).max() * noise
    return {"zero": np.zeros(s.n_nodes), "one_cycle": u1, "rough": rough}


def check_steps(S, s, lev, F, eta, inner, label, ratios):
    Fd = dev(F)
    for start, u0 in starts(s, lev, F, eta).items():
        u_ref = u0.copy()
        for _ in range(inner):
            u_ref = mg.mg_cycle(lev, 0, u_ref, F, nu1=2, nu2=1, eta=eta, order="color4")
        u = dev(u0)
        S.cycles(Fd, u, 1, precision="mixed")
        got = host(u)
        tol, e = fp32_step_tolerance(s, F, u0, u_ref, cycles=inner)
        ratios.append(float((np.abs(got - u_ref) / tol)[s.dof].max()))
        assert_nodewise(got, u_ref, tol, (label, start, inner))
        # the step did the work: it moved u by the oracle's correction
        assert np.abs(got - u0).max() >= 0.5 * np.abs(e).max()


@pytest.mark.parametrize("fuse", [0, -1], ids=["fused", "separate"])
@pytest.mark.parametrize("eta", [4, 0])
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_mixed_step_iterates(name, eta, fuse, oracle_cache):
    from paper_2505_05105_gb300 import ghostmg as G
    p, s, lev, F = oracle_for(name, oracle_cache)
    ratios = []
    for inner in (1, 2):
        with G.Solver(dev(p.psi), p.N, p.x0, p.y0, p.h, precision="mixed", eta=eta,
                      inner=inner, fuse_max_tiles=fuse) as S:
            check_steps(S, s, lev, F, eta, inner, (name, eta, fuse), ratios)
    print(f"{name} eta={eta} fuse={fuse}: worst |diff| / bound {max(ratios):.3g}")


def test_separate_kernels_change_nothing_but_rounding():
    """The fused and the separate intermediate-level kernels run the same
    arithmetic; one refinement step agrees between them to the fp32 bound
    (not bit for bit: the fused step's restriction sums in another order)."""
    from paper_2505_05105_gb300 import ghostmg as G
    p = wl.flower(512, k=7, phase=0.3)
    s = gf.assemble_problem(p)
    F = s.rhs(p.f, p.g)
    out = []
    for fuse in (0, -1):
        with G.Solver(dev(p.psi), p.N, p.x0, p.y0, p.h, precision="mixed",
                      fuse_max_tiles=fuse) as S:
            u = torch.zeros(s.n_nodes, dtype=torch.float64, device="cuda")
            S.cycles(dev(F), u, 2, precision="mixed")
            out.append(host(u))
    scale = np.abs(out[0]).max()
    assert np.abs(out[0] - out[1]).max() <= 1e-5 * scale
