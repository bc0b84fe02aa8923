"""GPU parity on the large workload: the union of three seeded discs minus a
small disc (several cut features), random Fourier f, g = 0, at 8192^2 cells
(the large configuration bench.py times), mixed precision and fp64.

The oracle cannot assemble this system in a test, so it checks sampled
nodes one by one, each from its own element matrices (Eq. disc_bil_form,
Eq. disc_rhs): the operator row and F at sampled vertices of cut cells,
interior nodes and nodes next to the small disc, and the oracle's residual
F_p - sum_q A_pq u_q of the GPU solution there, within the solve's
tolerance (as tests/test_gpu_fullsize.py).  The mixed and fp64 solutions,
both stopped at 1e-10, agree to the accuracy the stopping test allows.
"""
import numpy as np
import pytest

from oracle import ghostfem as gf
from paper_2505_05105_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N = 8192


@pytest.fixture(scope="module")
def large():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2505_05105_gb300 import ghostmg as G
    G.load()
    p = wl.three_discs(N, seed=0)
    psi_s = gf.snap(p.psi, p.h, 1.75)
    return dict(G=G, p=p, psi_s=psi_s, cls=gf.cell_classes(psi_s))


def cell_matrices(L, cache, ic, jc):
    key = (ic, jc)
    if key in cache:
        return cache[key]
    p, cls = L["p"], L["cls"]
    c = cls[jc, ic]
    if c == gf.EXTERNAL:
        v = None
    elif c == gf.INTERNAL:
        S_int, M_int = cache.setdefault("interior", gf.interior_cell_matrices(p.h))
        v = (S_int, M_int, np.zeros((4, 4)))
    else:
        cc = gf.cut_cell(gf.cell_corner_psi(L["psi_s"], ic, jc), ic, jc, p.x0, p.y0, p.h, 2.0)
        v = (cc.Ke, cc.Mk, cc.Gk)
    cache[key] = v
    return v


def oracle_row(L, cache, i, j):
    p = L["p"]
    row = np.zeros(9)
    F = 0.0
    for dy in (0, 1):
        for dx in (0, 1):
            ic, jc = i - 1 + dx, j - 1 + dy
            if ic < 0 or jc < 0 or ic >= N or jc >= N:
                continue
            m = cell_matrices(L, cache, ic, jc)
            if m is None:
                continue
            Ke, Mk, Gk = m
            a = (i - ic) + 2 * (j - jc)
            for b in range(4):
                ni, nj = ic + (b & 1), jc + (b >> 1)
                row[(ni - i + 1) + 3 * (nj - j + 1)] += Ke[a, b]
                F += Mk[a, b] * p.f[nj, ni] + Gk[a, b] * p.g[nj, ni]
    return row, F


def sample_nodes(L, rng):
    cls, p = L["cls"], L["p"]
    jc, ic = np.nonzero(cls == gf.CUT)
    pick = rng.choice(len(ic), 80, replace=False)
    nodes = {(int(ic[k]) + dx, int(jc[k]) + dy) for k in pick for dx in (0, 1) for dy in (0, 1)}
    # nodes near the small disc cut out of the first disc
    c = np.array(p.meta["centres"][0])
    i0, j0 = ((c - np.array([p.x0, p.y0])) / p.h).astype(int)
    r = int(0.06 / p.h)
    for t in range(24):
        a = 2 * np.pi * t / 24
        nodes.add((int(i0 + r * np.cos(a)), int(j0 + r * np.sin(a))))
    jj, ii = np.nonzero(cls != gf.EXTERNAL)
    pick = rng.choice(len(ii), 120, replace=False)
    nodes |= {(int(ii[k]), int(jj[k])) for k in pick}
    return sorted(nodes)


def test_large_rows_rhs_and_solutions(large):
    G, p = large["G"], large["p"]
    rng = np.random.default_rng(31)
    nodes = sample_nodes(large, rng)
    cache = {}
    ref = {nd: oracle_row(large, cache, *nd) for nd in nodes}
    k = np.array([i + j * (N + 1) for i, j in nodes])
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()
    sols = {}
    for prec in ("mixed", "fp64"):
        with G.Solver(dev(p.psi), p.N, p.x0, p.y0, p.h, precision=prec) as S:
            if prec == "mixed":
                A0 = S.stencil(0)
                scale = max(np.abs(r).max() for r, _ in ref.values())
                for t, nd in enumerate(nodes):
                    assert np.abs(A0[k[t]] - ref[nd][0]).max() <= 1e-13 * scale, nd
                del A0
                F = torch.zeros((N + 1) ** 2, dtype=torch.float64, device="cuda")
                S.rhs(dev(p.f), dev(p.g), F)
                Fmax = float(F.abs().max())
                Fh = F[torch.from_numpy(k).cuda()].cpu().numpy()
                Fref = np.array([ref[nd][1] for nd in nodes])
                assert np.abs(Fh - Fref).max() <= 1e-13 * Fmax
                del F
            u = torch.zeros((N + 1) ** 2, dtype=torch.float64, device="cuda")
            info = S.solve(dev(p.f), dev(p.g), u, tol=1e-10)
            assert info.rel_res <= 1e-10
            uh = u.cpu().numpy().reshape(N + 1, N + 1)
            sols[prec] = uh
        for t, (i, j) in enumerate(nodes):
            row, Fp = ref[(i, j)]
            nb = np.array([uh[j + dj, i + di] for dj in (-1, 0, 1) for di in (-1, 0, 1)])
            r = Fp - float(np.dot(row, nb))
            slack = 1e-13 * (np.abs(row) @ np.abs(nb) + abs(Fp) + Fmax) + \
                1e-12 * scale * np.abs(nb).max()
            assert abs(r) <= 1e-10 * Fmax + slack, (prec, i, j, r)
    # both stopped at 1e-10: they agree to what the stopping test allows
    # (the Poisson problem's conditioning, ~N^2 in the max norm)
    diff = np.abs(sols["mixed"] - sols["fp64"]).max()
    assert diff <= 1e-10 * N * N * np.abs(sols["fp64"]).max() / 16, diff
