"""The largest grid the library accepts (n_cells = 32768: 1.07e9 nodes,
13 levels) on the GPU: the flower level set, setup, a mixed-precision solve
to 1e-10, and the oracle's residual of the solution at sampled nodes (rows
and F computed node by node from the oracle's element matrices, as in
tests/test_gpu_fullsize.py), within the solve's tolerance.
"""
import numpy as np
import pytest

from oracle import ghostfem as gf
from paper_2505_05105_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N = 32768


def test_largest_grid():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2505_05105_gb300 import ghostmg as G
    G.load()
    p = wl.flower(N)
    psi_s = gf.snap(p.psi, p.h, 1.75)
    cls = gf.cell_classes(psi_s)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()
    rng = np.random.default_rng(51)
    jc, ic = np.nonzero(cls == gf.CUT)
    pick = rng.choice(len(ic), 24, replace=False)
    nodes = sorted({(int(ic[k]) + dx, int(jc[k]) + dy) for k in pick
                    for dx in (0, 1) for dy in (0, 1)})
    # interior nodes along a line through the flower's centre
    nodes += [(N // 2 + d, N // 2 + d // 3) for d in range(-3000, 3001, 500)]
    cache = {}

    def cell(ic_, jc_):
        if (ic_, jc_) not in cache:
            c = cls[jc_, ic_]
            if c == gf.EXTERNAL:
                cache[(ic_, jc_)] = None
            elif c == gf.INTERNAL:
                S_int, M_int = gf.interior_cell_matrices(p.h)
                cache[(ic_, jc_)] = (S_int, M_int, np.zeros((4, 4)))
            else:
                cc = gf.cut_cell(gf.cell_corner_psi(psi_s, ic_, jc_), ic_, jc_, p.x0, p.y0,
                                 p.h, 2.0)
                cache[(ic_, jc_)] = (cc.Ke, cc.Mk, cc.Gk)
        return cache[(ic_, jc_)]

    ref = {}
    for (i, j) in nodes:
        row, F = np.zeros(9), 0.0
        for dy in (0, 1):
            for dx in (0, 1):
                m = cell(i - 1 + dx, j - 1 + dy)
                if m is None:
                    continue
                Ke, Mk, Gk = m
                a = (1 - dx) + 2 * (1 - dy)
                for b in range(4):
                    ni, nj = i - 1 + dx + (b & 1), j - 1 + dy + (b >> 1)
                    row[(ni - i + 1) + 3 * (nj - j + 1)] += Ke[a, b]
                    F += Mk[a, b] * p.f[nj, ni] + Gk[a, b] * p.g[nj, ni]
        ref[(i, j)] = (row, F)
    f, g = dev(p.f), dev(p.g)
    del psi_s, cls
    with G.Solver(dev(p.psi), N, p.x0, p.y0, p.h, precision="mixed") as S:
        n_levels, ndof, ncut, _ = S.counts()
        assert n_levels == 13 and ndof > 3e8
        u = torch.zeros_like(f)
        info = S.solve(f, g, u, tol=1e-10)
        assert info.rel_res <= 1e-10
        F = torch.zeros_like(f)
        S.rhs(f, g, F)
        Fmax = float(F.abs().max())
        del F
    W = N + 1
    idx = torch.tensor([(j + dj) * W + (i + di) for (i, j) in nodes
                        for dj in (-1, 0, 1) for di in (-1, 0, 1)], device="cuda")
    nb_all = u[idx].cpu().numpy().reshape(len(nodes), 9)
    scale = max(np.abs(r).max() for r, _ in ref.values())
    for t, nd in enumerate(nodes):
        row, Fp = ref[nd]
        nb = nb_all[t]
        r = Fp - float(np.dot(row, nb))
        slack = 1e-13 * (np.abs(row) @ np.abs(nb) + abs(Fp) + Fmax) + \
            1e-12 * scale * np.abs(nb).max()
        assert abs(r) <= 1e-10 * Fmax + slack, (nd, r)
    print(f"N={N}: {ndof} DOFs, {ncut} cut cells, {info.cycles} cycles, "
          f"{info.solve_ms:.1f} ms, setup {info.setup_ms:.0f} ms")
