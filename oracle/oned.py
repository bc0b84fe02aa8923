"""Oracle: the one-dimensional ghost-FEM multigrid of Sec. 4 (test
infrastructure only).

Plain fp64 restatement of the 1D model of Sec. 4 of Dilip & Coco,
"Multigrid methods for the ghost finite element approximation of elliptic
problems" (arXiv 2505.05105): Omega_art = [0, 1] with n cells of side
h = 1/n, Omega = (a, b), a = (1 - theta_1) h, b = 1 - (1 - theta_2) h; P1 hat
functions phi_0..phi_n (all of them belong to active cells); Dirichlet data
at a imposed by Nitsche's terms with penalty lambda (outward normal -1),
Neumann data at b (outward normal +1).  Eq. ls1dA / Eq. ls1dF print the
resulting matrices; here they are assembled from the element integrals of
Eq. disc_bil_form / Eq. disc_rhs so the printed forms can pin the assembly.

Multigrid (Sec. 3, Sec. 4.1-4.3): lexicographic Gauss-Seidel (P = L_h),
restriction Eq. resop (coarse hat = 1/2 phi_{2i-1} + phi_{2i} +
1/2 phi_{2i+1}), prolongation its transpose, Galerkin coarse operators
(Eq. galerkin read as R A P), coarsest grid h = 2^-3 solved exactly; the
two-grid correction scheme of Alg. 1 and the V- and W-cycles of Sec. 3.2.
The convergence factor follows Sec. 4.5: homogeneous problem, u^(0) = 1,
rho = mean of ||r^(m)||_inf / ||r^(m-1)||_inf over m = 41..50.

Stabilisation (Sec. 4.4): the local 2 x 2 pencil on the cut cell [x_0, x_1]
and the global pencil over V_h, both taken modulo constants (the rank-based
definition), give C = 1 / (theta_1 h).

Readings: the source enters through the P1
interpolant of nodal f (F^I = M f, M the mass on Omega); Eq.
shape_fun_relation's indices are off by one and are read as
1/2 phi_{2i-1} + phi_{2i} + 1/2 phi_{2i+1}; the snapping threshold written
h^{-alpha} is h^alpha (with the parameters of Sec. 4.5, theta_1 h > h^2, so
it never acts: the 1D routines take theta_1, theta_2 in (0, 1] as given).

Pins (tests/test_oracle_oned.py): Eq. ls1dA / Eq. ls1dF entry by entry;
the proposition of Sec. 4.2 (the splitting strategy's coarse residual equals
R r_h); the Galerkin operator equals the coarse grid's direct assembly with
theta -> (1 + theta) / 2 (Sec. 4.3); C = 1 / (theta_1 h) for the local and
the global pencils (Sec. 4.4, Sec. 4.5); dense solve = converged cycles; the
qualitative convergence findings of Sec. 4.5.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg

_GL_T, _GL_W = np.polynomial.legendre.leggauss(4)


@dataclass
class Problem1D:
    n: int
    theta1: float
    theta2: float
    lam: float

    @property
    def h(self):
        return 1.0 / self.n

    @property
    def a(self):
        return (1.0 - self.theta1) * self.h

    @property
    def b(self):
        return 1.0 - (1.0 - self.theta2) * self.h


def hat(i, x, n):
    """phi_i(x) and phi_i'(x) (one-sided inside a cell) on the grid of n cells."""
    h = 1.0 / n
    t = (x - i * h) / h
    v = np.where(np.abs(t) < 1.0, 1.0 - np.abs(t), 0.0)
    d = np.where((t > -1.0) & (t <= 0.0), 1.0 / h, np.where((t > 0.0) & (t < 1.0), -1.0 / h, 0.0))
    return v, d


def _cell_rule(lo, hi):
    x = lo + (hi - lo) * 0.5 * (_GL_T + 1.0)
    return x, 0.5 * (hi - lo) * _GL_W


def assemble(p: Problem1D):
    """The pieces of Eq. disc_bil_form / Eq. disc_rhs in 1D:
      S_ij = int_Omega phi_i' phi_j',   M_ij = int_Omega phi_i phi_j,
      A = S + lam phi(a) phi(a)^T + phi(a) phi'(a)^T + phi'(a) phi(a)^T
          (Nitsche terms at a, outward normal -1: lam u v - (n u') v - (n v') u),
      F = M f + gD g_a + gN g_b, gD = lam phi(a) + phi'(a), gN = phi(b).
    Returned as a dict with S, M, A, gD, gN, and the boundary vectors
    va = phi(a), da = phi'(a) (slopes of the cell that contains a)."""
    n, h = p.n, p.h
    S = np.zeros((n + 1, n + 1))
    M = np.zeros((n + 1, n + 1))
    for k in range(n):
        lo, hi = max(k * h, p.a), min((k + 1) * h, p.b)
        if hi <= lo:
            continue
        x, w = _cell_rule(lo, hi)
        for i in (k, k + 1):
            vi, di = hat(i, x, n)
            for j in (k, k + 1):
                vj, dj = hat(j, x, n)
                S[i, j] += np.sum(w * di * dj)
                M[i, j] += np.sum(w * vi * vj)
    k = min(int(np.floor(p.a / h)), n - 1)      # the cell [x_k, x_k+1] holding a
    va = np.zeros(n + 1)
    da = np.zeros(n + 1)
    va[k], va[k + 1] = 1.0 - (p.a - k * h) / h, (p.a - k * h) / h
    da[k], da[k + 1] = -1.0 / h, 1.0 / h
    A = S + p.lam * np.outer(va, va) + np.outer(va, da) + np.outer(da, va)
    gN = np.array([float(hat(i, np.array([p.b]), n)[0][0]) for i in range(n + 1)])
    return dict(S=S, M=M, A=A, gD=p.lam * va + da, gN=gN, va=va, da=da)


def printed_system(p: Problem1D):
    """A_h = A^I + A^B + (A^B)^T + A^lambda and the vectors F^B / F^lambda /
    F^N per unit data, entry by entry as printed in Eq. ls1dA / Eq. ls1dF."""
    n, h, t1, t2, lam = p.n, p.h, p.theta1, p.theta2, p.lam
    AI = np.zeros((n + 1, n + 1))
    for i in range(1, n):
        AI[i, i] = 2.0
        AI[i, i - 1] = AI[i - 1, i] = -1.0
    AI[0, 0], AI[0, 1], AI[1, 0], AI[1, 1] = t1, -t1, -t1, 1.0 + t1
    AI[n - 1, n - 1], AI[n - 1, n], AI[n, n - 1], AI[n, n] = 1.0 + t2, -t2, -t2, t2
    AI /= h
    AB = np.zeros((n + 1, n + 1))
    AB[0, 0], AB[0, 1], AB[1, 0], AB[1, 1] = -t1, t1, t1 - 1.0, 1.0 - t1
    AB /= h
    Al = np.zeros((n + 1, n + 1))
    Al[0, 0], Al[0, 1], Al[1, 0], Al[1, 1] = t1 ** 2, t1 * (1 - t1), t1 * (1 - t1), (1 - t1) ** 2
    Al *= lam
    FB = np.zeros(n + 1)
    FB[0], FB[1] = -1.0 / h, 1.0 / h
    Fl = np.zeros(n + 1)
    Fl[0], Fl[1] = lam * t1, lam * (1 - t1)
    FN = np.zeros(n + 1)
    FN[n - 1], FN[n] = 1 - t2, t2
    ABN = np.zeros((n + 1, n + 1))
    ABN[n - 1, n - 1], ABN[n - 1, n], ABN[n, n - 1], ABN[n, n] = 1 - t2, t2 - 1, t2, -t2
    ABN /= h
    return dict(AI=AI, AB=AB, Al=Al, A=AI + AB + AB.T + Al, FB=FB, Fl=Fl, FN=FN, ABN=ABN)


def restriction(n: int) -> np.ndarray:
    """Eq. resop: (n/2 + 1) x (n + 1), rows 1/2 (1, 2, 1) around 2i."""
    R = np.zeros((n // 2 + 1, n + 1))
    for i in range(n // 2 + 1):
        R[i, 2 * i] = 1.0
        if 2 * i - 1 >= 0:
            R[i, 2 * i - 1] = 0.5
        if 2 * i + 1 <= n:
            R[i, 2 * i + 1] = 0.5
    return R


def split_coarse_residual(p: Problem1D, u, f, g_a, g_b):
    """r^SPLIT_2h of Eq. rsplit: R r^I_h (Eq. rhI) plus the boundary parts
    rebuilt on the coarse grid with theta -> (1 + theta) / 2 from the
    boundary residuals r_a = g_a - u(a), r_b = g_b - u'(b)."""
    n, h = p.n, p.h
    P = printed_system(p)
    FI = assemble(p)["M"] @ f
    rI = FI - P["AI"] @ u - P["AB"] @ u - P["ABN"] @ u
    t1, t2 = p.theta1, p.theta2
    ua = t1 * u[0] + (1 - t1) * u[1]
    dub = (u[n] - u[n - 1]) / h
    ra, rb = g_a - ua, g_b - dub
    m = n // 2
    r = restriction(n) @ rI
    r[0] += -ra / (2 * h) + 0.5 * p.lam * (t1 + 1) * ra
    r[1] += ra / (2 * h) + 0.5 * p.lam * (1 - t1) * ra
    r[m - 1] += 0.5 * (1 - t2) * rb
    r[m] += 0.5 * (t2 + 1) * rb
    return r


@dataclass
class Level1D:
    n: int
    A: np.ndarray
    R: np.ndarray = None     # to the next coarser level


def hierarchy(p: Problem1D, coarsest: int = 8):
    A = assemble(p)["A"]
    levels = [Level1D(p.n, A)]
    while levels[-1].n > coarsest:
        L = levels[-1]
        L.R = restriction(L.n)
        levels.append(Level1D(L.n // 2, L.R @ L.A @ L.R.T))
    return levels


def gs_lex(A, u, F):
    """One lexicographic Gauss-Seidel sweep (P = L_h, Sec. 4.1)."""
    for i in range(len(u)):
        u[i] += (F[i] - A[i] @ u) / A[i, i]
    return u


def cycle(levels, l, u, F, nu1=2, nu2=1, gamma_star=1, two_grid=False):
    """Alg. 1 on level l; the coarse equation solved exactly on the coarsest
    level, or at once below the finest level (two-grid scheme), else by
    gamma_star recursive cycles from zero (Sec. 3.2)."""
    L = levels[l]
    if l == len(levels) - 1:
        return np.linalg.solve(L.A, F)
    for _ in range(nu1):
        gs_lex(L.A, u, F)
    rc = L.R @ (F - L.A @ u)
    if two_grid:
        ec = np.linalg.solve(levels[l + 1].A, rc)
    else:
        ec = np.zeros_like(rc)
        for _ in range(gamma_star):
            ec = cycle(levels, l + 1, ec, rc, nu1, nu2, gamma_star)
    u += L.R.T @ ec
    for _ in range(nu2):
        gs_lex(L.A, u, F)
    return u


def convergence_factor(p: Problem1D, scheme="two-grid", cycles=50, first=41, nu1=2, nu2=1,
                       coarsest=8, u0=None):
    """Sec. 4.5: f = g_a = g_b = 0, u^(0) = 1 (or u0), rho = mean of the
    residual ratios for m = first..cycles.  scheme: "two-grid", "V" or "W"."""
    levels = hierarchy(p, coarsest)
    A = levels[0].A
    F = np.zeros(p.n + 1)
    u = np.ones(p.n + 1) if u0 is None else np.array(u0, dtype=np.float64)
    rn = [np.abs(F - A @ u).max()]
    for _ in range(cycles):
        u = cycle(levels, 0, u, F, nu1, nu2, gamma_star=2 if scheme == "W" else 1,
                  two_grid=scheme == "two-grid")
        rn.append(np.abs(F - A @ u).max())
    rho = [rn[m] / rn[m - 1] for m in range(first, cycles + 1)]
    return float(np.mean(rho)), rn


def local_C(p: Problem1D) -> float:
    """The 2 x 2 pencil of Sec. 4.4 on the cut cell [x_0, x_1] with
    K_ij = phi_i'(a) phi_j'(a), M_ij = int_a^{x_1} phi_i' phi_j', modulo
    the constants (both annihilate them; rank-based definition): the
    quotient of the one remaining direction (-1, 1)."""
    h, a = p.h, p.a
    d = np.array([-1.0 / h, 1.0 / h])           # slopes of phi_0, phi_1 on [x_0, x_1]
    K = np.outer(d, d)
    M = (h - a) * np.outer(d, d)
    v = np.array([-1.0, 1.0])
    return float(v @ K @ v / (v @ M @ v))


def global_C(p: Problem1D) -> float:
    """Sec. 4.5 / Sec. 5.2: the largest generalized eigenvalue of
    K v = Lambda M v over V_h, K_ij = phi_i'(a) phi_j'(a) (n = -1, squared),
    M_ij = int_Omega phi_i' phi_j', modulo constants (M + w w^T, w = 1/|1|,
    as for the 2D global constant)."""
    E = assemble(p)
    K = np.outer(E["da"], E["da"])
    m = p.n + 1
    w = np.full(m, 1.0 / np.sqrt(m))
    ev = scipy.linalg.eigh(K, E["S"] + np.outer(w, w), eigvals_only=True)
    return float(ev[-1])
