"""GPU parity at the benchmark's full size (flower, 4096 x 4096 cells,
5,022,066 DOFs), in the solver configuration bench.py times (default
parameters, mixed precision, adaptive residual checks).

Here the oracle computes sampled outputs one by one, each from its own
element matrices (Eq. disc_bil_form, Eq. disc_rhs):
  * cut cells: C(K), lambda_K, Ke, Mk, Gk of sampled cut cells;
  * operator rows and F at sampled nodes (vertices of cut cells, interior
    nodes, nodes on 64 x 32 tile edges), summed from the adjacent cells;
  * the GPU solution: the oracle's residual F_p - sum_q A_pq u_q at the
    sampled nodes is within the solve's tolerance;
The operators of every level, fp64 V-cycle iterates and mixed-precision
refinement steps at this size are compared with the whole oracle in
test_gpu_fullsize_oracle.py.
Tolerances as in test_gpu_parity.py: 1e-13 of the largest entry for rows
and element data (the same exact integrals in a different order).
"""
import numpy as np
import pytest

from oracle import ghostfem as gf
from paper_2505_05105_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N = 4096


@pytest.fixture(scope="module")
def full():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2505_05105_gb300 import ghostmg as G
    G.load()
    p = wl.flower(N)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()
    psi_s = gf.snap(p.psi, p.h, 1.75)
    cls = gf.cell_classes(psi_s)
    S = G.Solver(dev(p.psi), p.N, p.x0, p.y0, p.h, precision="mixed")
    out = dict(G=G, p=p, S=S, psi_s=psi_s, cls=cls, dev=dev)
    yield out
    S.close()


def cell_matrices(full, cache, ic, jc):
    """(Ke, Mk, Gk) of cell (ic, jc) from the oracle, None if external."""
    key = (ic, jc)
    if key in cache:
        return cache[key]
    p, cls = full["p"], full["cls"]
    c = cls[jc, ic]
    if c == gf.EXTERNAL:
        v = None
    elif c == gf.INTERNAL:
        S_int, M_int = cache.setdefault("interior", gf.interior_cell_matrices(p.h))
        v = (S_int, M_int, np.zeros((4, 4)))
    else:
        cc = gf.cut_cell(gf.cell_corner_psi(full["psi_s"], ic, jc), ic, jc, p.x0, p.y0, p.h, 2.0)
        v = (cc.Ke, cc.Mk, cc.Gk)
    cache[key] = v
    return v


def oracle_row(full, cache, i, j):
    """9-point row of node (i, j) (s = (di+1) + 3 (dj+1)) and F_(i,j)."""
    p = full["p"]
    row = np.zeros(9)
    F = 0.0
    for dy in (0, 1):
        for dx in (0, 1):
            ic, jc = i - 1 + dx, j - 1 + dy
            if ic < 0 or jc < 0 or ic >= N or jc >= N:
                continue
            m = cell_matrices(full, cache, ic, jc)
            if m is None:
                continue
            Ke, Mk, Gk = m
            a = (i - ic) + 2 * (j - jc)            # local vertex of (i, j)
            for b in range(4):
                ni, nj = ic + (b & 1), jc + (b >> 1)
                row[(ni - i + 1) + 3 * (nj - j + 1)] += Ke[a, b]
                F += Mk[a, b] * p.f[nj, ni] + Gk[a, b] * p.g[nj, ni]
    return row, F


def sample_nodes(full, rng):
    cls = full["cls"]
    jc, ic = np.nonzero(cls == gf.CUT)
    pick = rng.choice(len(ic), 60, replace=False)
    bnd = {(int(ic[k]) + dx, int(jc[k]) + dy) for k in pick for dx in (0, 1) for dy in (0, 1)}
    act = np.zeros((N + 1, N + 1), dtype=bool)
    jj, ii = np.nonzero(cls != gf.EXTERNAL)
    for dx in (0, 1):
        for dy in (0, 1):
            act[jj + dy, ii + dx] = True
    nj, ni = np.nonzero(act)
    pick = rng.choice(len(ni), 120, replace=False)
    inner = {(int(ni[k]), int(nj[k])) for k in pick}
    edge = [(i, j) for i, j in zip(ni[::997], nj[::997])
            if i % 64 in (0, 63) or j % 32 in (0, 31)][:40]
    return sorted(bnd | inner | set(edge))


def test_cut_cells_fullsize(full):
    rng = np.random.default_rng(11)
    cells, data = full["S"].cut_cells()
    assert len(cells) == 14918
    cache = {}
    for t in rng.choice(len(cells), 80, replace=False):
        c = int(cells[t])
        ic, jc = c % N, c // N
        cc = gf.cut_cell(gf.cell_corner_psi(full["psi_s"], ic, jc), ic, jc, full["p"].x0,
                         full["p"].y0, full["p"].h, 2.0)
        d = data[t]
        assert d[0] == pytest.approx(cc.C, rel=1e-13)
        assert d[1] == pytest.approx(cc.lam, rel=1e-13)
        for off, ref in ((4, cc.Ke), (20, cc.Mk), (36, cc.Gk)):
            got = d[off:off + 16].reshape(4, 4)
            assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
        cache[(ic, jc)] = (cc.Ke, cc.Mk, cc.Gk)


def test_rows_rhs_solution_fullsize(full):
    rng = np.random.default_rng(12)
    S, p, dev = full["S"], full["p"], full["dev"]
    nodes = sample_nodes(full, rng)
    cache = {}
    ref = {nd: oracle_row(full, cache, *nd) for nd in nodes}
    k = np.array([i + j * (N + 1) for i, j in nodes])
    # operator rows of level 0
    A0 = S.stencil(0)
    scale = max(np.abs(r).max() for r, _ in ref.values())
    for t, nd in enumerate(nodes):
        assert np.abs(A0[k[t]] - ref[nd][0]).max() <= 1e-13 * scale, nd
    # F = M f + G g
    F = torch.zeros((N + 1) ** 2, dtype=torch.float64, device="cuda")
    S.rhs(dev(p.f), dev(p.g), F)
    Fh = F[torch.from_numpy(k).cuda()].cpu().numpy()
    Fmax = float(F.abs().max())
    Fref = np.array([ref[nd][1] for nd in nodes])
    assert np.abs(Fh - Fref).max() <= 1e-13 * Fmax
    # the solution as bench.py computes it (mixed, default parameters) and in
    # fp64: the oracle's residual at the sampled nodes is within tol
    for prec in ("mixed", "fp64"):
        Sx = S if prec == "mixed" else full["G"].Solver(dev(p.psi), p.N, p.x0, p.y0, p.h,
                                                         precision="fp64")
        u = torch.zeros_like(F)
        info = Sx.solve(dev(p.f), dev(p.g), u, tol=1e-10)
        assert info.rel_res <= 1e-10
        uh = u.cpu().numpy().reshape(N + 1, N + 1)
        for t, (i, j) in enumerate(nodes):
            row, Fp = ref[(i, j)]
            nb = np.array([uh[j + dj, i + di] for dj in (-1, 0, 1) for di in (-1, 0, 1)])
            r = Fp - float(np.dot(row, nb))
            # rounding of both evaluations, and the row / F differences
            # bounded above (1e-13 of the largest entry)
            slack = 1e-13 * (np.abs(row) @ np.abs(nb) + abs(Fp) + Fmax) + \
                1e-12 * scale * np.abs(nb).max()
            assert abs(r) <= 1e-10 * Fmax + slack, (prec, i, j, r)
        if Sx is not S:
            Sx.close()
