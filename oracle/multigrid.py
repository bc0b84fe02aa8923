"""Oracle: geometric multigrid for the ghost-FEM system (test infrastructure only).

Plain fp64 restatement of Sec. 3 (Alg. 1 two-grid correction scheme, V- and
W-cycles, convergence factor), Sec. 4.1-4.3 (Gauss-Seidel smoother,
R = P^T, Galerkin coarse operator, Eq. galerkin) and Sec. 5.1 (bilinear
transfer between Omega_h and Omega_2h) and Sec. 5.3 (eta extra smoothing
iterations on the cut cells).

Readings:
* Eq. galerkin is read as A_2h = R A_h P with R = P^T (as printed it is not
  conformable); P is bilinear interpolation, rows restricted to fine DOFs.
* A coarse node is a DOF iff its column of P is non-zero.  A coarse cell is
  internal if its four children are, external if its four children are, and
  "cut" otherwise; cut nodes of a level are the vertices of its cut cells.
* Gauss-Seidel order: ``lex`` is the lexicographic order of the node index
  k = i + j (n+1) (P = L_h, Sec. 4.1); ``color4`` visits the four classes
  (i mod 2, j mod 2) in the order (0,0), (1,0), (0,1), (1,1).  Same-colour
  nodes never share a 9-point stencil, so ``color4`` is Gauss-Seidel for the
  colour-permuted matrix.
* One smoothing step = one sweep over all DOFs, then eta sweeps over the cut
  nodes of that level in the same order (Sec. 5.3); applied on every
  non-coarsest level.
* The coarsest level (8 x 8 cells unless told otherwise) is solved exactly.
* With strong Dirichlet box sides the box nodes of every level are not DOFs
  (P has no columns for the coarse ones).
* Coarse re-discretisation (the alternative to Eq. galerkin the paper
  describes in Sec. 4.3 / Sec. 5): level l is assembled from scratch on its
  own grid (h_l = 2^l h) from the level set sampled at its nodes, snapped with
  h_l^alpha, with its own cut cells and lambda_K = gamma C(K); its DOFs are
  the vertices of its own active cells; P and R = P^T as before.
* Stop when ||F - A u||_inf / ||F||_inf <= tol.

Pins (tests/test_oracle_multigrid.py): the printed n = 2 restriction matrix
(Sec. 5.1); the Galerkin operator equals direct assembly of a_h on coarse hat
functions; dense brute force = sparse direct = converged V-cycle at 8..16
cells; convergence factor rho ~ 0.1 with gamma = 2, eta = 4 (Sec. 5.3).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .ghostfem import CUT, EXTERNAL, INTERNAL, System


def interp_1d(nc: int) -> sp.csr_matrix:
    """Linear interpolation from nc+1 coarse to 2nc+1 fine nodes (Sec. 4.2:
    the coarse hat is 1/2 phi_{2i-1} + phi_{2i} + 1/2 phi_{2i+1})."""
    nf = 2 * nc
    r, c, v = [], [], []
    for i in range(nc + 1):
        r.append(2 * i); c.append(i); v.append(1.0)
        for d in (-1, 1):
            if 0 <= 2 * i + d <= nf:
                r.append(2 * i + d); c.append(i); v.append(0.5)
    return sp.csr_matrix((v, (r, c)), shape=(nf + 1, nc + 1))


def prolongation(nc: int, dof_fine: np.ndarray | None = None) -> sp.csr_matrix:
    """Bilinear interpolation (Sec. 5.1) from (nc+1)^2 coarse nodes to
    (2nc+1)^2 fine nodes, node index k = i + j (n+1); rows of fine nodes that
    are not DOFs are zero."""
    p1 = interp_1d(nc)
    P = sp.kron(p1, p1, format="csr")     # row (j, i) = j*(nf+1) + i
    if dof_fine is not None:
        P = sp.diags(dof_fine.astype(np.float64)) @ P
    return P.tocsr()


def coarse_cell_classes(cls: np.ndarray) -> np.ndarray:
    n = cls.shape[0] // 2
    c = cls.reshape(n, 2, n, 2).transpose(0, 2, 1, 3).reshape(n, n, 4)
    out = np.full((n, n), CUT, dtype=np.int64)
    out[(c == INTERNAL).all(-1)] = INTERNAL
    out[(c == EXTERNAL).all(-1)] = EXTERNAL
    return out


def cut_node_mask(cls: np.ndarray) -> np.ndarray:
    n = cls.shape[0]
    m = np.zeros((n + 1, n + 1), dtype=bool)
    jj, ii = np.nonzero(cls == CUT)
    for dj in (0, 1):
        for di in (0, 1):
            m[jj + dj, ii + di] = True
    return m.ravel()


@dataclass
class Level:
    n: int                       # cells per side
    A: sp.csr_matrix             # (n+1)^2 square
    dof: np.ndarray              # bool (n+1)^2
    cls: np.ndarray              # (n, n)
    cut_nodes: np.ndarray        # bool (n+1)^2
    P: sp.csr_matrix | None = None    # from level below (coarser) to this one
    _cache: dict | None = None

    def colour_of(self):
        j, i = np.divmod(np.arange((self.n + 1) ** 2), self.n + 1)
        return (i % 2) + 2 * (j % 2)


def build_hierarchy(system: System, coarsest: int = 8, rediscretise_psi=None) -> list[Level]:
    """Levels 0 (fine) .. L (n = coarsest) with Galerkin operators
    A_{l+1} = P_l^T A_l P_l (Eq. galerkin, read as R A P), or, given the
    fine grid's nodal level set (before snapping) as rediscretise_psi, with
    every coarse level assembled from scratch on its own grid."""
    lev = [Level(system.N, system.A.tocsr(), system.dof.copy(), system.cls.copy(),
                 cut_node_mask(system.cls))]
    step = 1
    while lev[-1].n > coarsest:
        f = lev[-1]
        nc = f.n // 2
        step *= 2
        P = prolongation(nc, f.dof)
        if system.box_strong:
            # the coarse box nodes are strong Dirichlet nodes too: their
            # corrections are zero
            jn, in_ = np.divmod(np.arange((nc + 1) ** 2), nc + 1)
            inner = ~((in_ == 0) | (jn == 0) | (in_ == nc) | (jn == nc))
            P = (P @ sp.diags(inner.astype(np.float64))).tocsr()
            P.eliminate_zeros()
        f.P = P
        if rediscretise_psi is None:
            Ac = (P.T @ f.A @ P).tocsr()
            Ac.eliminate_zeros()
            dofc = np.asarray(abs(P).sum(axis=0)).ravel() > 0
            clsc = coarse_cell_classes(f.cls)
            lev.append(Level(nc, Ac, dofc, clsc, cut_node_mask(clsc) & dofc))
        else:
            from .ghostfem import assemble
            psi = np.asarray(rediscretise_psi, dtype=np.float64).reshape(system.N + 1,
                                                                        system.N + 1)
            sc = assemble(psi[::step, ::step], nc, system.x0, system.y0, system.h * step,
                          system.gamma, system.alpha, box_strong=system.box_strong)
            lev.append(Level(nc, sc.A.tocsr(), sc.dof.copy(), sc.cls.copy(),
                             cut_node_mask(sc.cls) & sc.dof))
    return lev


# ----------------------------------------------------------------------------
# Gauss-Seidel smoother (Sec. 4.1) and extra cut-cell sweeps (Sec. 5.3)
# ----------------------------------------------------------------------------

def _prep(L: Level):
    if L._cache is not None:
        return L._cache
    col = L.colour_of()
    diag = L.A.diagonal()
    c = {"diag": diag}
    for name, mask in (("all", L.dof), ("cut", L.cut_nodes & L.dof)):
        groups = []
        for k in range(4):
            idx = np.flatnonzero(mask & (col == k))
            groups.append((idx, L.A[idx]))
        c["c4_" + name] = groups
        idx = np.flatnonzero(mask)
        Asub = L.A[idx][:, idx]
        c["lex_" + name] = (idx, sp.tril(Asub, format="csr"))
    L._cache = c
    return c


def gs_sweep(L: Level, u, F, subset="all", order="color4"):
    """One Gauss-Seidel sweep u <- u + P^{-1}(F - A u) with P the lower
    triangle (incl. diagonal) of A in the chosen order, restricted to the
    nodes of ``subset`` ('all' DOFs or 'cut' nodes); the others stay fixed."""
    c = _prep(L)
    if order == "color4":
        for idx, Ar in c["c4_" + subset]:
            if len(idx):
                u[idx] += (F[idx] - Ar @ u) / c["diag"][idx]
    elif order == "lex":
        idx, Lo = c["lex_" + subset]
        if len(idx):
            r = (F - L.A @ u)[idx]
            u[idx] += spla.spsolve_triangular(Lo, r, lower=True)
    else:
        raise ValueError(order)
    return u


def smooth(L: Level, u, F, eta, order):
    gs_sweep(L, u, F, "all", order)
    for _ in range(eta):
        gs_sweep(L, u, F, "cut", order)
    return u


def gs_sweep_backward(L: Level, u, F, subset="all"):
    """The transpose of gs_sweep(order="color4") as an approximate inverse:
    the same colour updates in the reverse colour order (1,1), (0,1), (1,0),
    (0,0) (each colour's update E D^{-1} E^T is symmetric, so reversing the
    sequence transposes the product)."""
    c = _prep(L)
    for idx, Ar in reversed(c["c4_" + subset]):
        if len(idx):
            u[idx] += (F[idx] - Ar @ u) / c["diag"][idx]
    return u


def smooth_transposed(L: Level, u, F, eta):
    """The transpose of one smoothing step (smooth with order="color4"): the
    eta cut-node sweeps first, then the full sweep, each backward."""
    for _ in range(eta):
        gs_sweep_backward(L, u, F, "cut")
    gs_sweep_backward(L, u, F, "all")
    return u


def coarse_solve(L: Level, F):
    """Exact solve on the DOFs of L (dense Cholesky when small, sparse LU
    otherwise, e.g. for the coarse grid of the two-grid scheme)."""
    d = np.flatnonzero(L.dof)
    u = np.zeros_like(F)
    if len(d) <= 2000:
        Ad = L.A[d][:, d].toarray()
        u[d] = scipy.linalg.cho_solve(scipy.linalg.cho_factor(Ad), F[d])
    elif len(d):
        u[d] = spla.spsolve(L.A[d][:, d].tocsc(), F[d])
    return u


def mg_cycle(levels, l, u, F, nu1=2, nu2=1, eta=4, order="color4", gamma_star=1,
             exact_below=None):
    """One multigrid cycle on level l (Alg. 1 applied recursively, Sec. 3.2):
    gamma_star = 1 is the V-cycle, 2 the W-cycle.  ``exact_below`` = l+1 turns
    it into the two-grid correction scheme."""
    L = levels[l]
    if l == len(levels) - 1:
        return coarse_solve(L, F)
    for _ in range(nu1):
        smooth(L, u, F, eta, order)
    r = F - L.A @ u
    Fc = L.P.T @ r
    if exact_below is not None and l + 1 >= exact_below:
        ec = coarse_solve(levels[l + 1], Fc)
    else:
        ec = np.zeros_like(Fc)
        for _ in range(gamma_star):
            ec = mg_cycle(levels, l + 1, ec, Fc, nu1, nu2, eta, order, gamma_star,
                          exact_below)
    u += L.P @ ec
    for _ in range(nu2):
        smooth(L, u, F, eta, order)
    return u


def mg_cycle_transposed(levels, l, u, F, nu1=2, nu2=1, eta=4):
    """The transposed V(nu1, nu2)-cycle.  A V-cycle is u <- u + B (F - A u)
    with B its approximate inverse (Alg. 1 applied recursively, Sec. 3.2);
    B is a product of symmetric steps (colour updates, the coarse correction
    P B_2h P^T with R = P^T, the exact coarsest solve), so B^T takes the same
    steps in the reverse order: nu2 transposed smoothing steps, the
    transposed cycle on the coarse level, nu1 transposed smoothing steps.
    Since A is symmetric, k of these from u = 0 give the transpose of k
    V-cycles from u = 0 (the adjoint of the iteration).  Pinned:
    tests/test_oracle_multigrid.py builds B and B^T column by column."""
    L = levels[l]
    if l == len(levels) - 1:
        return coarse_solve(L, F)
    for _ in range(nu2):
        smooth_transposed(L, u, F, eta)
    r = F - L.A @ u
    Fc = L.P.T @ r
    ec = mg_cycle_transposed(levels, l + 1, np.zeros_like(Fc), Fc, nu1, nu2, eta)
    u += L.P @ ec
    for _ in range(nu1):
        smooth_transposed(L, u, F, eta)
    return u


def residual(L: Level, u, F):
    r = F - L.A @ u
    r[~L.dof] = 0.0
    return r


def solve(levels, F, u0=None, tol=1e-10, max_cycles=100, **kw):
    """Cycles from u0 (default 0) until ||F - A u||_inf / ||F||_inf <= tol.
    Returns (u, history of relative residuals, cycles)."""
    L = levels[0]
    u = np.zeros_like(F) if u0 is None else np.array(u0, dtype=np.float64)
    u[~L.dof] = 0.0
    nF = np.abs(F).max()
    hist = [np.abs(residual(L, u, F)).max() / nF]
    k = 0
    while hist[-1] > tol and k < max_cycles:
        u = mg_cycle(levels, 0, u, F, **kw)
        k += 1
        hist.append(np.abs(residual(L, u, F)).max() / nF)
    return u, hist, k


def convergence_factor(levels, cycles=30, first=21, two_grid=False, **kw):
    """rho = mean of ||r^(m)||_inf / ||r^(m-1)||_inf for m = first..cycles on the
    homogeneous problem with u^(0) = 1 on the DOFs (Sec. 3.1, Sec. 5.3)."""
    L = levels[0]
    F = np.zeros((L.n + 1) ** 2)
    u = L.dof.astype(np.float64)
    rn = [np.abs(residual(L, u, F)).max()]
    for _ in range(cycles):
        u = mg_cycle(levels, 0, u, F, exact_below=1 if two_grid else None, **kw)
        rn.append(np.abs(residual(L, u, F)).max())
    rho = [rn[m] / rn[m - 1] for m in range(first, cycles + 1)]
    return float(np.mean(rho)), rn
