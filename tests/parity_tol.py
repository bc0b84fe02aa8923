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
U32 = 2.0 ** -24        # unit roundoff of fp32

# Row data: both sides integrate the same exact element integrals (Eq.
# disc_bil_form) with different quadrature and summation orders.  On the cut
# cells the Nitsche terms cancel (a penalty term of size ~gamma C(K) |Gamma|
# against the normal-derivative terms), so an entry is only defined to a few
# hundred ulp of the largest entry of its row; the operator-row tests hold
# every row to ROW_REL of its own largest entry.  A relative change delta of
# node p's row moves a Gauss-Seidel update, and the exact solution at a node
# whose equation is dominated by its own row, by delta S_p (first order): the
# data term of the node-wise bounds.  It matters only at weak ghost nodes
# (S_p up to 1e6 |u|, below); elsewhere S_p ~ 2 |u| and it is ~1e-12 |u|.
ROW_REL = 2e-13
# Coarse rows are Galerkin sums P^T A P of up to 81 fine contributions each
# (Eq. galerkin), with the same cancellation compounded (row-relative
# differences up to ~3e-11 on the 8 x 8 level at 4096^2); they are held to
# 1e-13 of their level's largest entry only, since they reach the node-wise
# bounds through the coarse-grid correction alone, whose effect on a fine
# iterate is smooth and covered by the rel max|u| term.

# Rounding events of one fp32 V(2,1)-cycle with eta = 4, per node of a level:
# (nu1 + nu2)(1 + eta) = 15 Gauss-Seidel updates, each with two fp32
# roundings of relative size U32 (the stored fp32 row coefficients and the
# update's own arithmetic), so about 32 U32 per cycle; twice that is the
# constant of the fp32 iterate bound.
C32 = 64


def sensitivity(system, F, u):
    A = system.A
    diag = A.diagonal()
    S = (np.abs(F) + abs(A) @ np.abs(u)) / np.where(diag > 0, diag, 1.0)
    S[~system.dof] = 0.0
    return S


def node_tolerance(system, F, u, rel, c):
    """rel max|u| + (c eps + ROW_REL) S_p: the benchmark spec bound, the
    rounding of c Gauss-Seidel updates and the row-data term."""
    return rel * np.abs(u).max() + (c * EPS + ROW_REL) * sensitivity(system, F, u)


def row_rel_diff(got_rows, ref_rows):
    """Per row: max |difference| / the reference row's largest entry (0 on
    empty rows)."""
    scale = np.abs(ref_rows).max(axis=1)
    d = np.abs(got_rows - ref_rows).max(axis=1)
    return np.where(scale > 0, d / np.where(scale > 0, scale, 1.0), d)


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
    node on a tiny cut triangle can reach 1e4-1e6 (its diagonal ~1e-12-1e-8
    against couplings ~1e-6-1e-4 to a heavily penalised neighbour).  Such
    "weak ghost nodes" (A_p > 100) are reported by the tests; their bound is
    the same as every other node's."""
    A = system.A
    diag = A.diagonal()
    off = abs(A) @ np.ones(A.shape[0]) - np.abs(diag)
    amp = off / np.where(diag > 0, diag, 1.0)
    amp[~system.dof] = 0.0
    return amp


def assert_solution(got, ref, system, F, rel, c=64, what=""):
    """Node-wise comparison of a converged solution with the exact one, at
    every DOF: rel max|u| + (c eps + ROW_REL) S_p + 2 |r_p| / a_pp (the
    the benchmark spec bound, rounding, the row-data term, and what the stopping
    residual leaves at a node dominated by its diagonal).  Returns the
    number of weak ghost nodes (A_p > 100) and the largest A_p."""
    tol = node_tolerance(system, F, ref, rel, c) + 2 * residual_term(system, F, got)
    assert_nodewise(got, ref, tol, what)
    amp = amplification(system)
    return int(((amp > 100) & system.dof).sum()), float(amp.max())


def correction_sensitivity(system, r, e):
    """S_p of the correction equation A e = r (the equation an fp32 V-cycle
    of the mixed-precision refinement solves): (|r_p| + sum_q |a_pq| |e_q|)
    / a_pp, in units of e."""
    A = system.A
    diag = A.diagonal()
    S = (np.abs(r) + abs(A) @ np.abs(e)) / np.where(diag > 0, diag, 1.0)
    S[~system.dof] = 0.0
    return S


def fp32_step_tolerance(system, F, u0, u_ref, cycles=1):
    """Node-wise bound for one mixed-precision refinement step from u0 (fp64
    residual r = F - A u0, `cycles` fp32 V-cycles on A e = sigma r from e = 0,
    fp64 update) against the fp64 oracle's V-cycles from the same u0, whose
    result u_ref = u0 + e with e the exact-arithmetic correction:
        C32 * cycles * U32 * (max|e| + S_p(e))  +  64 eps S_p(u_ref)
    The first term is the fp32 arithmetic of the cycles (relative to the
    correction, which sets their scale through sigma); the second the fp64
    residual and update (with the row-data term)."""
    e = u_ref - u0
    r = F - system.A @ u0
    r[~system.dof] = 0.0
    S_e = correction_sensitivity(system, r, e)
    return (C32 * cycles * U32 * (np.abs(e).max() + S_e)
            + (64 * EPS + ROW_REL) * sensitivity(system, F, u_ref)), e
