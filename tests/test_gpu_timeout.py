"""Failure detection on the GPU without a GPU fault: every wait a kernel of
the library makes (the completion of its shared-memory tensor and bulk
copies) is bounded.  With the poll budget set to zero (mg_set_wait_limit)
each such wait gives up at once: the kernel records the timeout, lets its
own copy land (a second wait with the default budget), and stops; the call
returns MG_ERR_TIMEOUT.  The GPU keeps answering: the same handle, with the
default budget again, and the next handle solve exactly as before."""
import numpy as np
import pytest

from paper_2505_05105_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_bounded_wait_runs_out_and_the_gpu_still_answers(precision):
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    from paper_2505_05105_gb300 import ghostmg as G
    p = wl.flower(256)
    f, g = dev(p.f), dev(p.g)
    with G.Solver(dev(p.psi), p.N, p.x0, p.y0, p.h, precision=precision) as S:
        ref = torch.zeros_like(f)
        S.solve(f, g, ref, tol=1e-11)
        G.mg_set_wait_limit(S.handle, 0)
        u = torch.zeros_like(f)
        with pytest.raises(G.GhostMGError) as exc:
            S.solve(f, g, u, tol=1e-11)
        assert exc.value.code == G.MG_ERR_TIMEOUT
        # the step-level call reports it too
        F = torch.zeros_like(f)
        S.rhs(f, g, F)
        with pytest.raises(G.GhostMGError) as exc:
            S.cycles(F, u, 1, precision=precision)
        assert exc.value.code == G.MG_ERR_TIMEOUT
        # default budget again: the same handle solves as before
        G.mg_set_wait_limit(S.handle, -1)
        u.zero_()
        info = S.solve(f, g, u, tol=1e-11)
        assert info.rel_res <= 1e-11
        assert torch.equal(u, ref)
    # and a new handle, and torch's own work, run normally
    with G.Solver(dev(p.psi), p.N, p.x0, p.y0, p.h, precision=precision) as S2:
        u2 = torch.zeros_like(f)
        S2.solve(f, g, u2, tol=1e-11)
        assert torch.equal(u2, ref)
    assert float((f * 2).sum()) == pytest.approx(2 * float(f.sum()))


def test_wait_limit_arguments():
    from paper_2505_05105_gb300 import ghostmg as G
    G.load()
    assert G.load().mg_set_wait_limit(None, 5) == G.MG_ERR_INVALID_ARG
    p = wl.circle64(64)
    with G.Solver(dev(p.psi), p.N, p.x0, p.y0, p.h) as S:
        assert G.load().mg_set_wait_limit(S.handle, 1 << 33) == G.MG_ERR_INVALID_ARG
        G.mg_set_wait_limit(S.handle, 1000)
        u = torch.zeros((p.N + 1) ** 2, dtype=torch.float64, device="cuda")
        S.solve(dev(p.f), dev(p.g), u, tol=1e-11)     # a short but sufficient budget
