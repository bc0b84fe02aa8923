"""Every GPU path of the library on small problems, for the bounds-checked
build (run as a child process by test_gpu_bounds.py, with GHOSTMG_CHECKED=1
for the checked library or unset for the normal one).

Prints one JSON object: the library's bounds-check state and, per workload,
the status and a checksum of its output (sum and sum of squares of the
result), so that the two builds can be compared.
"""
import json
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_2505_05105_gb300 import ghostmg as G  # noqa: E402
from paper_2505_05105_gb300 import workloads as wl  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


def checksum(t):
    torch.cuda.synchronize()
    a = t.detach().double().cpu().numpy().ravel()
    return [float(np.sum(a)), float(np.sum(a * a))]


def solver(p, **kw):
    return G.Solver(dev(p.psi), p.N, p.x0, p.y0, p.h, **kw)


def run():
    out = {}

    def record(name, fn):
        try:
            out[name] = {"status": G.MG_OK, "sum": fn()}
        except G.GhostMGError as e:
            out[name] = {"status": e.code, "sum": None}

    def solve(p, tol=1e-10, **kw):
        def fn():
            S = solver(p, **kw)
            u = torch.zeros((p.N + 1) ** 2, dtype=torch.float64, device="cuda")
            gN = dev(p.gN) if getattr(p, "gN", None) is not None and "neumann_mask" in kw else None
            S.solve(dev(p.f), dev(p.g), u, tol=tol, gN=gN)
            S.close()
            return checksum(u)
        return fn

    c64, f128, f512 = wl.circle64(64), wl.flower(128, k=7, phase=0.3), wl.flower(512, k=7)
    f2048 = wl.flower(2048)
    record("circle64_fp64", solve(c64, tol=1e-12))
    record("circle64_global", solve(c64, tol=1e-12, c_global=0))
    record("flower128_w", solve(f128, cycle="W"))
    record("flower128_twogrid", solve(f128, cycle="two-grid"))
    record("flower128_rediscretise", solve(f128, coarse="rediscretise"))
    for fm in (0, -1):
        for eta in (4, 0):
            record(f"flower512_mixed_fuse{fm}_eta{eta}",
                   solve(f512, precision="mixed", fuse_max_tiles=fm, eta=eta))
    record("flower2048_mixed", solve(f2048, precision="mixed"))
    record("flower2048_fp64", solve(f2048, precision="fp64"))
    an = wl.annulus(64)
    record("annulus64_neumann", solve(an, tol=1e-12, neumann_mask=an.neumann_mask))
    rc = wl.rectangle(64, 0.37)
    record("rectangle64_box", solve(rc, tol=1e-12, box_sides=True))

    def adjoint():
        S = solver(f128)
        u = torch.zeros((f128.N + 1) ** 2, dtype=torch.float64, device="cuda")
        S.solve(dev(f128.f), dev(f128.g), u, tol=1e-12)
        dLdf, dLdg = torch.zeros_like(u), torch.zeros_like(u)
        S.adjoint(dev(wl.adjoint_target(f128, 1)), dLdf, dLdg)
        F = torch.zeros_like(u)
        S.rhs(dev(f128.f), dev(f128.g), F)
        w = torch.zeros_like(u)
        S.cycles_transposed(F, w, 3)
        rmax, _ = S.residual(F, u)
        S.close()
        return checksum(dLdf) + checksum(dLdg) + checksum(w) + [rmax]
    record("flower128_adjoint", adjoint)

    def static_residual():
        S = solver(c64)
        u = dev(np.linspace(0.0, 1.0, (c64.N + 1) ** 2))
        F = torch.zeros_like(u)
        S.rhs(dev(c64.f), dev(c64.g), F)
        r = torch.zeros_like(u)
        G.mg_residual_static(S.handle, F, u, r)
        S.close()
        return checksum(r)
    record("circle64_residual_static", static_residual)

    def batch():
        ps = [wl.batch_geometry(i, seed=5, sizes=(16, 32, 64, 128)) for i in range(6)]
        ps += [wl.batch_geometry(0, seed=6, sizes=(256,))]
        with G.BatchSolver(ps) as B:
            f, g = dev(B.pack([p.f for p in ps])), dev(B.pack([p.g for p in ps]))
            u = torch.zeros(B.total, dtype=torch.float64, device="cuda")
            B.solve(f, g, u, tol=1e-10)
            return checksum(u)
    record("batch7", batch)

    def oned():
        probs = [(64, 0.3, 0.01, 1.1 / (0.3 / 64)), (128, 0.05, 0.01, 128.0 ** 2)]
        total = sum(n + 1 for n, *_ in probs)
        u = torch.ones(total, dtype=torch.float64, device="cuda")
        G.mg1d_cycles(probs, u, cycle="V", cycles=5)
        return checksum(u)
    record("oned", oned)

    enabled, hits = G.mg_bounds_check()
    return {"checked": enabled, "hits": hits, "runs": out}


if __name__ == "__main__":
    print(json.dumps(run()))
