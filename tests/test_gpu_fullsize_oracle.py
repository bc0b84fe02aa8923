"""GPU parity at the benchmark's full size (flower, 4096 x 4096 cells,
5,022,066 DOFs) against the whole oracle: the oracle assembles the system
(Eq. disc_bil_form, Eq. disc_rhs) and its Galerkin hierarchy (Eq. galerkin,
R = P^T, Sec. 5.1) at this size (about half a minute and 9 GB of host memory),
and the GPU's operators of every level, the first fp64 V-cycles and the first
mixed-precision refinement steps -- in the launch configuration bench.py
times (mixed precision, default parameters: the fine fp32 sweep, the
separate fp32 kernels with the prolongation added on load on level 1, the
fused steps on levels 2-5, the tail) -- are compared with it node by node.

Tolerances: rows of every level to 1e-13 of the level's largest entry and
each row to ROW_REL of its own largest entry; fp64 iterates after k cycles
to 1e-10 max|u| + (64 k eps + ROW_REL) S_p (tests/parity_tol.py: the
row-data term matters at the weak ghost nodes, A_p up to 1.2e6 here); a
mixed step to tests/parity_tol.fp32_step_tolerance (fp32 rounding of the
correction).
"""
import numpy as np
import pytest

from oracle import ghostfem as gf
from oracle import multigrid as mg
from paper_2505_05105_gb300 import workloads as wl
from parity_tol import (ROW_REL, assert_nodewise, fp32_step_tolerance, node_tolerance,
                        row_rel_diff)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N = 4096


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.fixture(scope="module")
def big():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2505_05105_gb300 import ghostmg as G
    G.load()
    p = wl.flower(N)
    s = gf.assemble_problem(p)
    lev = mg.build_hierarchy(s)
    F = s.rhs(p.f, p.g)
    S = G.Solver(dev(p.psi), p.N, p.x0, p.y0, p.h, precision="mixed")
    yield dict(p=p, s=s, lev=lev, F=F, S=S)
    S.close()


def test_rows_every_level_fullsize(big):
    from test_gpu_parity import oracle_rows
    S, lev = big["S"], big["lev"]
    assert S.counts()[0] == len(lev)
    for l, L in enumerate(lev):
        got = S.stencil(l)
        ref = oracle_rows(L.A, L.n)
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err <= 1e-13, (l, L.n, err)
        rr = row_rel_diff(got, ref)
        print(f"4096^2 level {l}: worst row-relative difference {rr.max():.3g}")
        if l == 0:
            assert rr.max() <= ROW_REL, (l, L.n, int(np.argmax(rr)), float(rr.max()))


def test_fp64_vcycle_iterates_fullsize(big):
    s, lev, F, S = big["s"], big["lev"], big["F"], big["S"]
    u_ref = np.zeros(s.n_nodes)
    u = torch.zeros(s.n_nodes, dtype=torch.float64, device="cuda")
    Fd = dev(F)
    for k in (1, 2):
        u_ref = mg.mg_cycle(lev, 0, u_ref, F, nu1=2, nu2=1, eta=4, order="color4")
        S.cycles(Fd, u, 1, precision="fp64")
        assert_nodewise(host(u), u_ref, node_tolerance(s, F, u_ref, 1e-10, 64 * k), ("fp64", k))


def test_mixed_steps_fullsize(big):
    s, lev, F, S = big["s"], big["lev"], big["F"], big["S"]
    u0 = np.zeros(s.n_nodes)
    Fd = dev(F)
    for step in (1, 2):
        u_ref = mg.mg_cycle(lev, 0, u0.copy(), F, nu1=2, nu2=1, eta=4, order="color4")
        u = dev(u0)
        S.cycles(Fd, u, 1, precision="mixed")
        got = host(u)
        tol, e = fp32_step_tolerance(s, F, u0, u_ref)
        ratio = float((np.abs(got - u_ref) / tol)[s.dof].max())
        print(f"4096^2 mixed step {step}: worst |diff| / bound {ratio:.3g}")
        assert_nodewise(got, u_ref, tol, ("mixed", step))
        u0 = u_ref
