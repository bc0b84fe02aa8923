"""The allocation-free residual (mg_residual_static) gives the same result as
mg_residual.  It exists for callers that cannot allocate device memory while
they use the solver (real-time loops that cannot take an allocation's
device-wide synchronisation, frameworks whose own allocator owns all device
memory); its reduction scratch is a fixed device array inside the library.
Two calls in a row with different inputs check that nothing stale leaks from
one call into the next.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2505_05105_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


def test_residual_static_matches_residual_twice():
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    from paper_2505_05105_gb300 import ghostmg as G
    p = wl.flower(128)
    with G.Solver(dev(p.psi), p.N, p.x0, p.y0, p.h) as S:
        n = (p.N + 1) ** 2
        F = torch.zeros(n, dtype=torch.float64, device="cuda")
        S.rhs(dev(p.f), dev(p.g), F)
        rng = np.random.default_rng(1)
        for trial in range(2):
            u = dev(rng.standard_normal(n) * (trial + 1))
            r_ref = torch.zeros(n, dtype=torch.float64, device="cuda")
            n_ref = S.residual(F, u, r_ref)
            r_new = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
            n_new = G.mg_residual_static(S.handle, F, u, r_new)
            torch.cuda.synchronize()
            a, b = r_ref.cpu().numpy(), r_new.cpu().numpy()
            scale = np.abs(a).max()
            assert np.abs(a - b).max() <= 1e-12 * scale, trial
            assert n_new[0] == pytest.approx(n_ref[0], rel=1e-12)
            assert n_new[1] == pytest.approx(n_ref[1], rel=1e-12)
        # norms only, r omitted
        n_only = G.mg_residual_static(S.handle, F, u)
        assert n_only == n_new
