"""Oracle adjoint (dL/df = M^T w, dL/dg = G^T w with A w = dL/du) pinned to
things it does not compute itself: central differences of the oracle's
forward solve (exact up to rounding for a quadratic loss, since u is affine
in f and g), and the structure of the gradients (zero off the DOFs; dL/dg
zero away from cut cells, where g does not enter F)."""
import numpy as np
import pytest

from oracle import ghostfem as gf
from paper_2505_05105_gb300 import workloads as wl


def loss_and_grad(system, u, ut, inside):
    r = (u - ut) * inside
    return 0.5 * float(r @ r), r


@pytest.mark.parametrize("make", [lambda: wl.circle64(16), lambda: wl.flower(32)])
def test_adjoint_matches_central_differences(make):
    p = make()
    s = gf.assemble_problem(p)
    rng = np.random.default_rng(3)
    inside = (np.ravel(p.psi) < 0).astype(float)
    ut = rng.standard_normal(s.n_nodes)
    f0, g0 = np.ravel(p.f).copy(), np.ravel(p.g).copy()

    def L(f, g):
        u = gf.direct_solve(s, s.rhs(f, g))
        return loss_and_grad(s, u, ut, inside)[0]

    u = gf.direct_solve(s, s.rhs(f0, g0))
    _, dLdu = loss_and_grad(s, u, ut, inside)
    dLdf, dLdg = gf.adjoint(s, dLdu)
    assert np.all(dLdf[~s.dof] == 0) and np.all(dLdg[~s.dof] == 0)
    # g enters F only through cut cells: dL/dg vanishes at nodes with no cut cell
    N = p.N
    cutnode = np.zeros((N + 1, N + 1), bool)
    jc, ic = np.nonzero(s.cls == gf.CUT)
    for dx in (0, 1):
        for dy in (0, 1):
            cutnode[jc + dy, ic + dx] = True
    assert np.all(dLdg[~cutnode.ravel()] == 0)
    dofs = np.flatnonzero(s.dof)
    cut = np.flatnonzero(cutnode.ravel())
    h = 1e-3
    scale = max(np.abs(dLdf).max(), np.abs(dLdg).max())
    for q in rng.choice(dofs, 12, replace=False):
        e = np.zeros_like(f0); e[q] = h
        fd = (L(f0 + e, g0) - L(f0 - e, g0)) / (2 * h)
        assert fd == pytest.approx(dLdf[q], abs=1e-9 * scale)
    for q in rng.choice(cut, 12, replace=False):
        e = np.zeros_like(g0); e[q] = h
        fd = (L(f0, g0 + e) - L(f0, g0 - e)) / (2 * h)
        assert fd == pytest.approx(dLdg[q], abs=1e-9 * scale)


def test_neumann_adjoint_matches_central_differences():
    """dL/dg_N = N^T w on the annulus (Neumann outer circle): central
    differences of the forward solve, zero away from the Neumann cut cells."""
    p = wl.annulus(32)
    s = gf.assemble_problem(p)
    rng = np.random.default_rng(4)
    inside = (np.ravel(p.psi) < 0).astype(float)
    ut = rng.standard_normal(s.n_nodes)
    f0, g0, n0 = (np.ravel(a).copy() for a in (p.f, p.g, p.gN))

    def L(gN):
        u = gf.direct_solve(s, s.rhs(f0, g0, gN))
        return loss_and_grad(s, u, ut, inside)[0]

    u = gf.direct_solve(s, s.rhs(f0, g0, n0))
    _, dLdu = loss_and_grad(s, u, ut, inside)
    dLdn = gf.adjoint_neumann(s, dLdu)
    N = p.N
    neu = np.zeros((N + 1, N + 1), bool)
    for c in s.cut:
        if c.neumann:
            neu[c.jc:c.jc + 2, c.ic:c.ic + 2] = True
    assert np.all(dLdn[~neu.ravel()] == 0) and np.abs(dLdn).max() > 0
    h = 1e-3
    scale = np.abs(dLdn).max()
    for q in rng.choice(np.flatnonzero(neu.ravel()), 12, replace=False):
        e = np.zeros_like(n0); e[q] = h
        fd = (L(n0 + e) - L(n0 - e)) / (2 * h)
        assert fd == pytest.approx(dLdn[q], abs=1e-9 * scale)


def test_box_adjoint_matches_central_differences():
    """With strong box sides g also enters F as - B g: dL/dg = G^T w - B^T w,
    nonzero on the box nodes next to the domain; central differences."""
    p = wl.rectangle(16, 0.37)
    s = gf.assemble_problem(p)
    rng = np.random.default_rng(5)
    inside = ((np.ravel(p.psi) < 0) & s.dof).astype(float)
    ut = rng.standard_normal(s.n_nodes)
    f0, g0 = np.ravel(p.f).copy(), np.ravel(p.g).copy()

    def L(g):
        u = gf.direct_solve(s, s.rhs(f0, g))
        return loss_and_grad(s, u, ut, inside)[0]

    u = gf.direct_solve(s, s.rhs(f0, g0))
    _, dLdu = loss_and_grad(s, u, ut, inside)
    _, dLdg = gf.adjoint(s, dLdu)
    ring = np.zeros((p.N + 1, p.N + 1), bool)
    ring[0, :] = ring[-1, :] = ring[:, 0] = ring[:, -1] = True
    assert np.abs(dLdg[ring.ravel()]).max() > 0
    scale = np.abs(dLdg).max()
    h = 1e-3
    for q in list(rng.choice(np.flatnonzero(ring.ravel() & (dLdg != 0)), 8, replace=False)) + \
            list(rng.choice(np.flatnonzero(dLdg != 0), 8, replace=False)):
        e = np.zeros_like(g0); e[q] = h
        fd = (L(g0 + e) - L(g0 - e)) / (2 * h)
        assert fd == pytest.approx(dLdg[q], abs=1e-9 * scale)

