"""Node-wise parity tolerances derived from the arithmetic.

Both sides compute in fp64, with the same exact integrals and stencils taken
in a different order, so the data agree to a few ulp.  A node's value is then
reproducible to about eps S_p, where

    S_p = (|F_p| + sum_q |a_pq| |u_q|) / a_pp

is the rounding sensitivity of node p's equation (a Gauss-Seidel update
divides a sum of that size by a_pp).  For ordinary nodes S_p ~ 2 |u| and the
fixed bound rel * max|u| dominates; S_p is large only at ghost nodes that
hang on a tiny cut region (a_pp ~ 1e-9 for a cut triangle of area ~1e-5 h^2,
which snapping with alpha = 1.75 still allows), where two correct fp64
evaluations cannot agree better than c eps S_p.  c counts the rounding
events a node goes through (about 30 Gauss-Seidel updates per V(2,1)-cycle
with eta = 4).
"""
import numpy as np

EPS = np.finfo(np.float64).eps


def sensitivity(system, F, u):
    A = system.A
    diag = A.diagonal()
    S = (np.abs(F) + abs(A) @ np.abs(u)) / np.where(diag > 0, diag, 1.0)
    S[~system.dof] = 0.0
    return S


def node_tolerance(system, F, u, rel, c):
    return rel * np.abs(u).max() + c * EPS * sensitivity(system, F, u)


def residual(system, F, u):
    """F - A u accumulated in long double (the oracle's own check)."""
    A = system.A.tocsr()
    r = F.astype(np.longdouble) - (A.astype(np.longdouble) @ u.astype(np.longdouble))
    r = np.asarray(r, dtype=np.float64)
    r[~system.dof] = 0.0
    return r


def residual_term(system, F, u):
    """Error a residual r_p implies at a node whose equation is dominated by
    its diagonal, |r_p| / a_pp (significant only where a_pp is tiny): a
    solution stopped on ||F - A u||_inf / ||F||_inf pins such nodes only that
    well."""
    diag = system.A.diagonal()
    return np.abs(residual(system, F, u)) / np.where(diag > 0, diag, 1.0)


def assert_nodewise(got, ref, tol, what=""):
    excess = np.abs(got - ref) - tol
    worst = int(np.argmax(excess))
    assert excess[worst] <= 0.0, (what, worst, float(np.abs(got - ref)[worst]), float(tol[worst]))


def amplification(system):
    """A_p = sum_{q != p} |a_pq| / a_pp: how much node p's equation amplifies
    errors of its neighbours.  It is O(1) for every internal node; a ghost
    node on a tiny cut triangle can reach 1e4-1e5 (its diagonal ~1e-8 against
    couplings ~1e-4 to a heavily penalised neighbour), so its computed value
    is only as good as its neighbours' values times A_p -- in any fp64
    implementation."""
    A = system.A
    diag = A.diagonal()
    off = abs(A) @ np.ones(A.shape[0]) - np.abs(diag)
    amp = off / np.where(diag > 0, diag, 1.0)
    amp[~system.dof] = 0.0
    return amp


def assert_solution(got, ref, system, F, rel, c=64, well_posed=100.0, what=""):
    """Node-wise comparison of a converged solution with the exact one:
    strict (rel max|u| + c eps S_p + 2 |r_p|/a_pp) on the well-posed nodes
    (A_p <= well_posed), and on the few weak ghost nodes the neighbours'
    worst error amplified by A_p (plus the same rounding and residual terms)."""
    tol = node_tolerance(system, F, ref, rel, c) + 2 * residual_term(system, F, got)
    amp = amplification(system)
    strong = amp <= well_posed
    err = np.abs(got - ref)
    assert_nodewise(np.where(strong, got, ref), ref, tol, (what, "well-posed nodes"))
    worst = err[strong].max() + rel * np.abs(ref).max()
    assert_nodewise(got, ref, tol + 4 * amp * worst, (what, "weak ghost nodes"))
    return int((~strong & system.dof).sum()), float(amp.max())
