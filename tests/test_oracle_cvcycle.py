"""The C restatement of the oracle's V-cycle (oracle/vcycle.c, the CPU
baseline bench.py times on the host cores) against oracle.multigrid: the
same colour-ordered Gauss-Seidel (Sec. 4.1), extra cut-cell sweeps
(Sec. 5.3), transfers (Sec. 5.1) and exact coarsest solve, so iterates
agree to rounding (the restriction sums in another order), on several
thread counts; and a solve reaches the oracle's direct solution."""
import numpy as np
import pytest

from oracle import cvcycle
from oracle import ghostfem as gf
from oracle import multigrid as mg
from paper_2505_05105_gb300 import workloads as wl


@pytest.fixture(scope="module")
def flower():
    p = wl.flower(128)
    s = gf.assemble_problem(p)
    lev = mg.build_hierarchy(s)
    return p, s, lev, s.rhs(p.f, p.g)


@pytest.mark.parametrize("eta, nu", [(4, (2, 1)), (0, (1, 1)), (2, (3, 0))])
@pytest.mark.parametrize("threads", [1, 3])
def test_iterates_match_oracle(flower, eta, nu, threads):
    p, s, lev, F = flower
    C = cvcycle.CVCycle(lev)
    u_ref = np.zeros(s.n_nodes)
    u = np.zeros(s.n_nodes)
    for k in range(1, 4):
        u_ref = mg.mg_cycle(lev, 0, u_ref, F, nu1=nu[0], nu2=nu[1], eta=eta, order="color4")
        C.cycles(F, u, 1, nu1=nu[0], nu2=nu[1], eta=eta, threads=threads)
        scale = np.abs(u_ref).max()
        assert np.abs(u - u_ref).max() <= 1e-12 * scale, (k, np.abs(u - u_ref).max() / scale)
    C.close()


def test_solve_reaches_direct_solution(flower):
    p, s, lev, F = flower
    C = cvcycle.CVCycle(lev)
    u, hist, k = C.solve(F, tol=1e-13, threads=2)
    assert 0 < k < 40 and hist[-1] <= 1e-13
    _, hist_py, k_py = mg.solve(lev, F, tol=1e-13)
    assert k == k_py                       # same cycle, same stopping test
    ud = gf.direct_solve(s, F)
    assert np.abs(u - ud).max() <= 1e-9 * np.abs(ud).max()
    assert cvcycle.CVCycle.threads(2) == 2
