"""Oracle: nodal ghost-FEM discretisation (test infrastructure only).

Plain fp64 restatement of Sec. 2 (Eq. Vhact, Eq. disc_bil_form, Eq. disc_rhs,
snapping back to grid) and Sec. 5.2 (cut configurations, cut lengths theta,
local stabilisation C(K), Eq. c_triangle, Eq. c_pentagon) of Dilip & Coco,
"Multigrid methods for the ghost finite element approximation of elliptic
problems" (arXiv 2505.05105).  Integrals are evaluated in cell-local
coordinates (relative to the cell's lower-left node, so thin cut regions lose
no digits to cancellation) with Gauss-Legendre rules far above the polynomial
degree of every integrand, so they are exact up to rounding.

Readings where the paper is silent or garbled:
* Snapping acts on nodal values: a node with -h^alpha < psi < 0 gets psi = 0.
* A node is internal iff psi < 0; psi = 0 counts as external (Sec. 5.2).
* A cell with two internal vertices on a diagonal (not covered by Sec. 5.2) is
  resolved with the bilinear centre value psi_c = mean of the four corners:
  psi_c < 0 gives one hexagon with two boundary segments, otherwise two
  disjoint triangles.  Zero-length boundary segments are dropped.
* h_K is the cell side h (the paper writes meas(K)).
* C(K) is the largest generalized eigenvalue of the local pencil of Sec. 5.2
  on the complement of constants (the rank-based definition of Sec. 4.4).
  Triangles use Eq. c_triangle (equal to that definition, pinned in tests);
  pentagons and hexagons use Eq. c_pentagon; quadrilaterals and the
  two-triangle saddle use the definition (the printed quadrilateral formula
  is garbled).
* f and g_D enter through their Q1 interpolants of nodal values, so
  F = M f + G g exactly (M: mass on the active region, G: boundary load).
* Mixed boundary conditions (Eq. poisson_model_prob with Gamma_N non-empty):
  each cut cell's piece of the boundary is wholly Dirichlet or wholly
  Neumann, as a per-cell mask says.  A Neumann cut cell contributes only its
  volume term to a_h (no Nitsche terms, Eq. disc_bil_form sums them over
  K cap Gamma_D) and its boundary mass to the load: with the Q1 interpolant
  of nodal g_N, int_{K cap Gamma_N} g_N phi_i = (Nk g_N)_i, Nk_ij =
  int_{K cap Gamma} phi_i phi_j (Eq. disc_rhs).  F = M f + G g_D + N g_N.

Pins (tests/test_oracle_*.py): Q1 stiffness closed form and stencil 8/3, -1/3;
the 1D matrices of Eq. ls1dA / ls1dF on a straight cut; Eq. c_triangle vs the
eigen definition; quad theta1 = theta2 => C = 1/(theta h) (Sec. 5.3);
polygon areas against closed forms and pi r^2; symmetry and positive
definiteness by dense eigenvalues; second-order convergence on manufactured
solutions; the adjoint gradients against central differences of the forward
solve (exact up to rounding for the quadratic losses used) and their support
(zero off the DOFs, dL/dg zero away from cut cells).  Neumann cells: a
straight cut reduces to the Neumann end of the 1D system (Eq. ls1dA, the
theta_2 block, and Eq. ls1dF, F^N); a patch test with a straight Neumann
side reproduces bilinear harmonic solutions exactly; second-order
convergence on the annulus with Dirichlet inner and Neumann outer circle
(Sec. 5.3) and on the leaf with mixed data.  The global constant of Sec. 5.2
(``global_C``): 1 / (theta h) on a straight cut through the box (the 1D value
of Sec. 4.4 carried over by the tensor-product structure), 1 / (min theta h)
on a strip with two cuts, at most the largest local C(K), 0 with every cut
cell Neumann (tests/test_oracle_global_lambda.py).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg
import scipy.sparse as sp

EXTERNAL, INTERNAL, CUT = 0, 1, 2

# local vertex order inside a cell: v0=(0,0) v1=(1,0) v2=(0,1) v3=(1,1)
LOCAL_REF = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0]])
# the same vertices walked counter-clockwise around the cell
CCW = (0, 1, 3, 2)

_GL_T, _GL_W = np.polynomial.legendre.leggauss(6)
GL_S = 0.5 * (_GL_T + 1.0)          # nodes on [0, 1]
GL_W = 0.5 * _GL_W                  # weights on [0, 1]


# ----------------------------------------------------------------------------
# Sec. 2: snapping back to grid, cell classes
# ----------------------------------------------------------------------------

def snap(psi: np.ndarray, h: float, alpha: float) -> np.ndarray:
    """Snapping back to grid (Sec. 2): a node x in Omega (psi < 0) with
    |psi(x)| < h^alpha gets psi(x) = 0."""
    out = np.array(psi, dtype=np.float64, copy=True)
    out[(out < 0.0) & (out > -(h ** alpha))] = 0.0
    return out


def cell_classes(psi_s: np.ndarray) -> np.ndarray:
    """Cell class by the number of internal vertices (Sec. 2, Sec. 5.2):
    4 internal -> INTERNAL, 0 -> EXTERNAL, otherwise CUT.  Shape (N, N),
    indexed [jc, ic]."""
    inside = (psi_s < 0.0).astype(np.int64)
    nin = inside[:-1, :-1] + inside[:-1, 1:] + inside[1:, :-1] + inside[1:, 1:]
    cls = np.full(nin.shape, CUT, dtype=np.int64)
    cls[nin == 4] = INTERNAL
    cls[nin == 0] = EXTERNAL
    return cls


def cell_corner_psi(psi_s: np.ndarray, ic: int, jc: int) -> np.ndarray:
    """psi at the local vertices v0..v3 of cell (ic, jc)."""
    return np.array([psi_s[jc, ic], psi_s[jc, ic + 1],
                     psi_s[jc + 1, ic], psi_s[jc + 1, ic + 1]])


# ----------------------------------------------------------------------------
# Sec. 5.2: cut configurations and cut lengths
# ----------------------------------------------------------------------------

@dataclass
class Piece:
    poly: np.ndarray                      # (m, 2) reference coords, CCW
    segments: list = field(default_factory=list)   # [(p, q)] reference coords


def cut_pieces(psi4):
    """Pieces of K cap Omega_h in reference coordinates of the cell.

    Walks the cell boundary counter-clockwise, keeping internal vertices and
    the linear-interpolation intersection point of every sign-changing edge,
    at distance theta h from the internal end with
    theta = psi_in / (psi_in - psi_out) (Sec. 5.2).  A boundary segment runs
    from each exit point to the following entry point, so its right-hand
    normal points out of Omega_h.

    Returns (config, pieces, thetas) with config one of 'internal',
    'external', 'triangle', 'quad', 'pentagon', 'hexagon', 'two_triangles'.
    """
    psi4 = np.asarray(psi4, dtype=np.float64)
    inside = psi4 < 0.0
    nin = int(inside.sum())
    if nin == 0:
        return "external", [], []
    if nin == 4:
        return "internal", [Piece(LOCAL_REF[list(CCW)].copy(), [])], []

    pts, kinds, thetas = [], [], []
    for a, b in zip(CCW, CCW[1:] + CCW[:1]):
        if inside[a]:
            pts.append(LOCAL_REF[a].copy())
            kinds.append("v")
        if inside[a] != inside[b]:
            i_in, i_out = (a, b) if inside[a] else (b, a)
            th = psi4[i_in] / (psi4[i_in] - psi4[i_out])
            thetas.append(th)
            pts.append(LOCAL_REF[i_in] + th * (LOCAL_REF[i_out] - LOCAL_REF[i_in]))
            kinds.append("exit" if inside[a] else "entry")

    def segs_of(idx):
        out = []
        m = len(idx)
        for t in range(m):
            p, q = idx[t], idx[(t + 1) % m]
            if kinds[p] == "exit" and kinds[q] == "entry":
                if not np.array_equal(pts[p], pts[q]):
                    out.append((pts[p], pts[q]))
        return out

    diagonal = nin == 2 and (inside[0] == inside[3])
    if not diagonal:
        config = {1: "triangle", 2: "quad", 3: "pentagon"}[nin]
        idx = list(range(len(pts)))
        return config, [Piece(np.array(pts), segs_of(idx))], thetas

    # two internal vertices on a diagonal: bilinear centre value decides
    if psi4.mean() < 0.0:
        idx = list(range(len(pts)))
        return "hexagon", [Piece(np.array(pts), segs_of(idx))], thetas
    pieces = []
    m = len(pts)
    for t in range(m):
        if kinds[t] == "v":
            idx = [(t - 1) % m, t, (t + 1) % m]      # entry, vertex, exit
            pieces.append(Piece(np.array([pts[k] for k in idx]), segs_of(idx)))
    return "two_triangles", pieces, thetas


def triangle_legs(psi4):
    """Cut lengths (theta1, theta2) of the two edges at the single internal
    vertex of a triangular cut cell (Sec. 5.2, theta = psi_in/(psi_in-psi_out))."""
    psi4 = np.asarray(psi4, dtype=np.float64)
    v = int(np.flatnonzero(psi4 < 0.0)[0])
    nbrs = {0: (1, 2), 1: (0, 3), 2: (0, 3), 3: (1, 2)}[v]
    return tuple(psi4[v] / (psi4[v] - psi4[w]) for w in nbrs)


# ----------------------------------------------------------------------------
# Quadrature in physical coordinates
# ----------------------------------------------------------------------------

def triangle_rule(A, B, C):
    """Collapsed (Duffy) tensor Gauss-Legendre rule on triangle ABC:
    x = A + s(1-t)(B-A) + s t (C-A), dx = |(B-A)x(C-A)| s ds dt.
    6x6 points: exact for polynomials of total degree <= 10."""
    A, B, C = (np.asarray(v, dtype=np.float64) for v in (A, B, C))
    jac = abs((B[0] - A[0]) * (C[1] - A[1]) - (B[1] - A[1]) * (C[0] - A[0]))
    s, t = np.meshgrid(GL_S, GL_S, indexing="ij")
    ws, wt = np.meshgrid(GL_W, GL_W, indexing="ij")
    u, v = s * (1 - t), s * t
    pts = A + u.reshape(-1, 1) * (B - A) + v.reshape(-1, 1) * (C - A)
    w = (jac * s * ws * wt).reshape(-1)
    return pts, w


def polygon_rule(poly):
    """Fan triangulation of a convex polygon from its first vertex."""
    P, W = [], []
    for k in range(1, len(poly) - 1):
        p, w = triangle_rule(poly[0], poly[k], poly[k + 1])
        P.append(p)
        W.append(w)
    if not P:
        return np.zeros((0, 2)), np.zeros(0)
    return np.concatenate(P), np.concatenate(W)


def segment_rule(p, q):
    """Gauss-Legendre on the straight segment p->q (exact to degree 11)."""
    p, q = np.asarray(p, float), np.asarray(q, float)
    L = float(np.hypot(*(q - p)))
    pts = p + GL_S.reshape(-1, 1) * (q - p)
    return pts, GL_W * L


def q1_shape(x, y, xc, yc, h):
    """Q1 shape functions of the cell with lower-left corner (xc, yc) and their
    physical gradients at points (x, y).  Returns phi (n, 4), grad (n, 4, 2)."""
    xi = (np.asarray(x) - xc) / h
    et = (np.asarray(y) - yc) / h
    phi = np.stack([(1 - xi) * (1 - et), xi * (1 - et), (1 - xi) * et, xi * et], -1)
    gx = np.stack([-(1 - et), (1 - et), -et, et], -1) / h
    gy = np.stack([-(1 - xi), -xi, (1 - xi), xi], -1) / h
    return phi, np.stack([gx, gy], -1)


# ----------------------------------------------------------------------------
# Element integrals of Eq. disc_bil_form / Eq. disc_rhs on one cell
# ----------------------------------------------------------------------------

@dataclass
class CellIntegrals:
    S: np.ndarray    # int_{K cap Omega} grad phi_i . grad phi_j
    Mp: np.ndarray   # int_{K cap Omega} phi_i phi_j
    Ms: np.ndarray   # int_{K cap Gamma} phi_i phi_j
    Bn: np.ndarray   # int_{K cap Gamma} (n . grad phi_j) phi_i
    Kn: np.ndarray   # int_{K cap Gamma} (n . grad phi_i)(n . grad phi_j)
    area: float
    length: float


def cell_integrals(pieces, xc, yc, h) -> CellIntegrals:
    S = np.zeros((4, 4)); Mp = np.zeros((4, 4)); Ms = np.zeros((4, 4))
    Bn = np.zeros((4, 4)); Kn = np.zeros((4, 4))
    area = 0.0; length = 0.0
    to_phys = lambda r: np.array([xc, yc]) + h * np.asarray(r, float)
    for pc in pieces:
        poly = np.array([to_phys(r) for r in pc.poly])
        X, W = polygon_rule(poly)
        if len(W):
            phi, g = q1_shape(X[:, 0], X[:, 1], xc, yc, h)
            S += np.einsum("q,qia,qja->ij", W, g, g)
            Mp += np.einsum("q,qi,qj->ij", W, phi, phi)
            area += W.sum()
        for (pr, qr) in pc.segments:
            p, q = to_phys(pr), to_phys(qr)
            d = q - p
            L = float(np.hypot(*d))
            n = np.array([d[1], -d[0]]) / L          # outward (right-hand) normal
            X, W = segment_rule(p, q)
            phi, g = q1_shape(X[:, 0], X[:, 1], xc, yc, h)
            dn = g @ n                                # (q, 4): n . grad phi
            Ms += np.einsum("q,qi,qj->ij", W, phi, phi)
            Bn += np.einsum("q,qj,qi->ij", W, dn, phi)
            Kn += np.einsum("q,qi,qj->ij", W, dn, dn)
            length += L
    return CellIntegrals(S, Mp, Ms, Bn, Kn, area, length)


# ----------------------------------------------------------------------------
# Sec. 4.4 / Sec. 5.2: stabilisation constant C(K)
# ----------------------------------------------------------------------------

_NULL1 = scipy.linalg.null_space(np.ones((1, 4)))   # basis of 1-perp in R^4


def c_definition(Kn, S) -> float:
    """Largest finite generalized eigenvalue of the local pencil K v = C M v
    (Sec. 5.2) with K = Kn, M = S given on the nodal basis.  Both annihilate
    constants, so the pencil is singular; following the rank-based
    definition (Sec. 4.4) the common null vector is deflated and the regular
    3x3 pencil is solved.  (Loses accuracy on thin cut regions, where the
    deflated nodal basis is ill conditioned; ``c_definition_pieces`` is the
    accurate form used by the assembly.)"""
    Kq = _NULL1.T @ Kn @ _NULL1
    Mq = _NULL1.T @ S @ _NULL1
    return float(scipy.linalg.eigh(Kq, Mq, eigvals_only=True)[-1])


def c_definition_pieces(pieces, xc, yc, h) -> float:
    """The same largest generalized eigenvalue, with Q1 modulo constants
    spanned by b1 = (x - xb)/s, b2 = (y - yb)/s, b3 = (x - xb)(y - yb)/s^2,
    (xb, yb) the area centroid of K cap Omega_h and s^2 its area.  Centring
    on the centroid makes the M-block diagonal, so the 3x3 pencil stays well
    conditioned for thin or small cut regions.
      M3_ab = int_{K cap Omega} grad b_a . grad b_b,
      K3_ab = int_{K cap Gamma} (n . grad b_a)(n . grad b_b)."""
    to_phys = lambda r: np.array([xc, yc]) + h * np.asarray(r, float)
    P, W = [], []
    for pc in pieces:
        X, w = polygon_rule(np.array([to_phys(r) for r in pc.poly]))
        P.append(X); W.append(w)
    X = np.concatenate(P); W = np.concatenate(W)
    area = W.sum()
    xb, yb = (W * X[:, 0]).sum() / area, (W * X[:, 1]).sum() / area
    sc = np.sqrt(area)

    def grads(x, y):      # (n, 3, 2)
        n = len(x)
        g = np.zeros((n, 3, 2))
        g[:, 0, 0] = 1.0 / sc
        g[:, 1, 1] = 1.0 / sc
        g[:, 2, 0] = (y - yb) / sc ** 2
        g[:, 2, 1] = (x - xb) / sc ** 2
        return g

    g = grads(X[:, 0], X[:, 1])
    M3 = np.einsum("q,qia,qja->ij", W, g, g)
    K3 = np.zeros((3, 3))
    for pc in pieces:
        for (pr, qr) in pc.segments:
            p, q = to_phys(pr), to_phys(qr)
            d = q - p
            n = np.array([d[1], -d[0]]) / np.hypot(*d)
            Xs, Ws = segment_rule(p, q)
            dn = grads(Xs[:, 0], Xs[:, 1]) @ n         # (n, 3)
            K3 += np.einsum("q,qi,qj->ij", Ws, dn, dn)
    return float(scipy.linalg.eigh(K3, M3, eigvals_only=True)[-1])


def c_triangle(theta1, theta2, h) -> float:
    """Eq. c_triangle: closed form of C for a triangular cut region whose legs
    along the cell edges are theta1 h and theta2 h."""
    t1, t2 = float(theta1), float(theta2)
    num = np.sqrt((t1 ** 2 + t2 ** 2) / t1 ** 2) * (
        3 * t1 ** 4 + 3 * t2 ** 4 + np.sqrt(3 * (t1 ** 8 + 10 * t1 ** 4 * t2 ** 4 + t2 ** 8)))
    return float(num / (h * t2 * (t1 ** 2 + t2 ** 2) ** 2))


def c_pentagon(h) -> float:
    """Eq. c_pentagon: the triangle value at theta1 = theta2 = 1, 3 sqrt(2)/h."""
    return 3.0 * np.sqrt(2.0) / h


def stabilisation_C(config, psi4, pieces, ints: CellIntegrals, xc, yc, h) -> float:
    if config == "triangle":
        return c_triangle(*triangle_legs(psi4), h)
    if config in ("pentagon", "hexagon"):
        return c_pentagon(h)
    if ints.length == 0.0:
        return 0.0
    return c_definition_pieces(pieces, xc, yc, h)


# ----------------------------------------------------------------------------
# One cut cell: element matrices of Eq. disc_bil_form and Eq. disc_rhs
# ----------------------------------------------------------------------------

@dataclass
class CutCell:
    ic: int
    jc: int
    config: str
    thetas: list
    C: float
    lam: float
    Ke: np.ndarray   # a_h element matrix
    Mk: np.ndarray   # mass on K cap Omega_h
    Gk: np.ndarray   # Dirichlet load: lam phi_i phi_j - (n.grad phi_i) phi_j
    ints: CellIntegrals
    neumann: bool = False
    Nk: np.ndarray = None   # Neumann load: phi_i phi_j on K cap Gamma_h


def cut_cell(psi4, ic, jc, x0, y0, h, gamma, neumann=False, c_global=None) -> CutCell:
    """Element matrices of cut cell (ic, jc).  The integrals are invariant
    under translation, so they are taken in cell-local coordinates (origin
    at the cell's lower-left corner, side h): absolute coordinates would add
    cancellation of order |x0 + ic h| / (size of the cut region).
    neumann: the cell's boundary piece belongs to Gamma_N.
    c_global: the global constant of Sec. 5.2 (``global_C``); when given,
    lambda = gamma c_global on every cut cell instead of gamma C(K)."""
    config, pieces, thetas = cut_pieces(psi4)
    ints = cell_integrals(pieces, 0.0, 0.0, h)
    C = stabilisation_C(config, psi4, pieces, ints, 0.0, 0.0, h)
    lam = gamma * (C if c_global is None else c_global)
    if neumann:
        # Eq. disc_bil_form has no boundary term on Gamma_N; Eq. disc_rhs
        # has int g_N phi_i over K cap Gamma_N
        return CutCell(ic, jc, config, thetas, C, lam, ints.S.copy(), ints.Mp.copy(),
                       np.zeros((4, 4)), ints, True, ints.Ms.copy())
    # a_h(phi_j, phi_i) on K: grad.grad + lam phi phi - (n.grad phi_j) phi_i
    #                          - (n.grad phi_i) phi_j           (Eq. disc_bil_form)
    Ke = ints.S + lam * ints.Ms - ints.Bn - ints.Bn.T
    # l_h with g_h = sum_j g_j phi_j: lam g phi_i - (n.grad phi_i) g  (Eq. disc_rhs)
    Gk = lam * ints.Ms - ints.Bn.T
    return CutCell(ic, jc, config, thetas, C, lam, Ke, ints.Mp.copy(), Gk, ints, False,
                   np.zeros((4, 4)))


def interior_cell_matrices(h):
    """Stiffness and mass of a whole cell, by the same quadrature."""
    ints = cell_integrals([Piece(LOCAL_REF[list(CCW)].copy(), [])], 0.0, 0.0, h)
    return ints.S, ints.Mp


# ----------------------------------------------------------------------------
# Global assembly
# ----------------------------------------------------------------------------

@dataclass
class System:
    N: int
    x0: float
    y0: float
    h: float
    gamma: float
    alpha: float
    psi_s: np.ndarray       # snapped nodal level set, (N+1, N+1)
    cls: np.ndarray         # cell classes, (N, N)
    dof: np.ndarray         # bool, (N+1)^2 flattened
    A: sp.csr_matrix        # (N+1)^2 square, zero rows/cols off the DOFs
    M: sp.csr_matrix
    G: sp.csr_matrix
    cut: list               # [CutCell]
    Gn: sp.csr_matrix = None   # Neumann load (None: all of Gamma is Dirichlet)
    B: sp.csr_matrix = None    # couplings of the DOFs to strong Dirichlet box nodes
    box_strong: bool = False

    @property
    def n_nodes(self):
        return (self.N + 1) ** 2

    def rhs(self, f, g, gN=None):
        """F = M f + G g_D (+ N g_N), Eq. disc_rhs with Q1 interpolants; with
        strong Dirichlet box sides also - B g (the box nodes' values g moved
        to the right-hand side)."""
        F = self.M @ np.ravel(f) + self.G @ np.ravel(g)
        if gN is not None and self.Gn is not None:
            F = F + self.Gn @ np.ravel(gN)
        if self.B is not None:
            F = F - self.B @ np.ravel(g)
        if self.box_strong:
            F[~self.dof] = 0.0
        return F


def cell_nodes(ic, jc, N):
    k0 = ic + jc * (N + 1)
    return np.array([k0, k0 + 1, k0 + N + 1, k0 + N + 2])


def assemble(psi, N, x0, y0, h, gamma=2.0, alpha=1.75, neumann_mask=None,
             box_strong=False, c_global=None) -> System:
    """A, M, G over all (N+1)^2 nodes (Eq. disc_bil_form, Eq. disc_rhs).
    neumann_mask: (N, N) cells [jc, ic], nonzero where a cut cell's boundary
    piece belongs to Gamma_N (ignored on other cells); None: all Dirichlet.
    box_strong: the nodes on the sides of the box (i or j equal to 0 or N)
    carry strong Dirichlet values (the rectangle of Sec. 5.3): they are not
    DOFs, and their couplings to the DOFs move to the right-hand side.
    c_global: lambda = gamma c_global on every cut cell (the global choice of
    Sec. 5.2) instead of the local lambda_K = gamma C(K)."""
    nm = None if neumann_mask is None else np.asarray(neumann_mask).reshape(N, N) != 0
    psi_s = snap(np.asarray(psi, dtype=np.float64).reshape(N + 1, N + 1), h, alpha)
    cls = cell_classes(psi_s)
    S_int, M_int = interior_cell_matrices(h)

    rows, cols, a_val, m_val, g_val, n_val = [], [], [], [], [], []
    jj, ii = np.nonzero(cls == INTERNAL)
    if len(ii):
        nodes = np.stack([cell_nodes(i, j, N) for i, j in zip(ii, jj)])   # (n, 4)
        rows.append(np.repeat(nodes, 4, axis=1).ravel())
        cols.append(np.tile(nodes, (1, 4)).ravel())
        a_val.append(np.tile(S_int.ravel(), len(ii)))
        m_val.append(np.tile(M_int.ravel(), len(ii)))
        g_val.append(np.zeros(16 * len(ii)))
        n_val.append(np.zeros(16 * len(ii)))
    cuts = []
    jj, ii = np.nonzero(cls == CUT)
    for i, j in zip(ii, jj):
        neu = bool(nm[j, i]) if nm is not None else False
        cc = cut_cell(cell_corner_psi(psi_s, i, j), int(i), int(j), x0, y0, h, gamma, neu,
                      c_global)
        cuts.append(cc)
        nodes = cell_nodes(i, j, N)
        rows.append(np.repeat(nodes, 4))
        cols.append(np.tile(nodes, 4))
        a_val.append(cc.Ke.ravel())
        m_val.append(cc.Mk.ravel())
        g_val.append(cc.Gk.ravel())
        n_val.append(cc.Nk.ravel())
    n = (N + 1) ** 2
    r = np.concatenate(rows) if rows else np.zeros(0, int)
    c = np.concatenate(cols) if cols else np.zeros(0, int)
    mk = lambda v: sp.csr_matrix((np.concatenate(v) if v else np.zeros(0), (r, c)), shape=(n, n))
    A, M, G = mk(a_val), mk(m_val), mk(g_val)
    Gn = mk(n_val) if nm is not None else None
    dof = np.zeros(n, dtype=bool)
    active = cls != EXTERNAL
    jj, ii = np.nonzero(active)
    for d in (0, 1, N + 1, N + 2):
        dof[ii + jj * (N + 1) + d] = True
    B = None
    if box_strong:
        jn, in_ = np.divmod(np.arange(n), N + 1)
        ring = (in_ == 0) | (jn == 0) | (in_ == N) | (jn == N)
        dof &= ~ring
        keep = sp.diags(dof.astype(np.float64))
        B = (keep @ A @ sp.diags(ring.astype(np.float64))).tocsr()
        B.eliminate_zeros()
        A = (keep @ A @ keep).tocsr()
        A.eliminate_zeros()
    return System(N, x0, y0, h, gamma, alpha, psi_s, cls, dof, A, M, G, cuts, Gn, B, box_strong)


def assemble_problem(prob, gamma=2.0, alpha=1.75, c_global=None) -> System:
    return assemble(prob.psi, prob.N, prob.x0, prob.y0, prob.h, gamma, alpha,
                    getattr(prob, "neumann_mask", None),
                    bool(getattr(prob, "meta", {}).get("box_strong", False)), c_global)


def global_C(psi, N, x0, y0, h, alpha=1.75, neumann_mask=None) -> float:
    """The global constant of Sec. 5.2: the largest generalized eigenvalue of
    K v = Lambda M v over the whole FE space, with
      K_ij = int_{Gamma_D} (n . grad phi_i)(n . grad phi_j) dS,
      M_ij = int_{Omega_h} grad phi_i . grad phi_j dx,
    both summed cell by cell from the same element integrals as the local
    pencil (K: the Dirichlet cut cells' Kn; M: every active cell's S).  Both
    annihilate the constants, so (rank-based definition, Sec. 4.4) the
    pencil is taken modulo constants: with w = 1 / |1|, every v = c 1 + v'
    with w . v' = 0 has the quotient of v', so max Lambda of (K, M + w w^T)
    is the same value, and M + w w^T is positive definite when the active
    region is connected.  Dense: for grids up to a few thousand DOFs."""
    psi_s = snap(np.asarray(psi, dtype=np.float64).reshape(N + 1, N + 1), h, alpha)
    cls = cell_classes(psi_s)
    nm = None if neumann_mask is None else np.asarray(neumann_mask).reshape(N, N) != 0
    S_int, _ = interior_cell_matrices(h)
    n = (N + 1) ** 2
    K = np.zeros((n, n))
    M = np.zeros((n, n))
    jj, ii = np.nonzero(cls != EXTERNAL)
    for i, j in zip(ii, jj):
        nodes = cell_nodes(i, j, N)
        if cls[j, i] == INTERNAL:
            M[np.ix_(nodes, nodes)] += S_int
            continue
        _, pieces, _ = cut_pieces(cell_corner_psi(psi_s, i, j))
        ints = cell_integrals(pieces, 0.0, 0.0, h)
        M[np.ix_(nodes, nodes)] += ints.S
        if nm is None or not nm[j, i]:
            K[np.ix_(nodes, nodes)] += ints.Kn
    dof = np.zeros(n, dtype=bool)
    for d in (0, 1, N + 1, N + 2):
        dof[ii + jj * (N + 1) + d] = True
    K = K[np.ix_(dof, dof)]
    M = M[np.ix_(dof, dof)]
    m = int(dof.sum())
    w = np.full(m, 1.0 / np.sqrt(m))
    ev = scipy.linalg.eigh(K, M + np.outer(w, w), eigvals_only=True,
                           subset_by_index=[m - 1, m - 1])
    return float(ev[-1])


def direct_solve(system: System, F: np.ndarray, refine: int = 4) -> np.ndarray:
    """Solution of A u = F on the DOFs (u = 0 elsewhere): sparse LU, then
    iterative refinement (Wilkinson) with the residual F - A u accumulated in
    extended precision (numpy longdouble), so the result is the exact
    solution rounded to fp64 even when cond(A) ~ 1e8 (small cut cells),
    where a plain fp64 solve is only good to about cond(A) eps."""
    import scipy.sparse.linalg as spla
    d = np.flatnonzero(system.dof)
    u = np.zeros(system.n_nodes)
    if len(d) == 0:
        return u
    A = system.A[d][:, d].tocsr()
    lu = spla.splu(A.tocsc())
    x = lu.solve(F[d])
    Al = sp.csr_matrix((A.data.astype(np.longdouble), A.indices, A.indptr), shape=A.shape)
    Fl = F[d].astype(np.longdouble)
    for _ in range(refine):
        r = Fl - Al @ x.astype(np.longdouble)
        dx = lu.solve(np.asarray(r, dtype=np.float64))
        x = np.asarray(x.astype(np.longdouble) + dx, dtype=np.float64)
        if np.abs(dx).max() <= 4 * np.finfo(np.float64).eps * np.abs(x).max():
            break
    u[d] = x
    return u


# ----------------------------------------------------------------------------
# Adjoint of the solve: gradients of a loss L(u) with respect to f and g
# ----------------------------------------------------------------------------

def adjoint(system: System, dLdu: np.ndarray):
    """dL/df and dL/dg (nodal vectors) of a loss L(u) where u solves
    A u = M f + G g on the DOFs (Eq. disc_bil_form, Eq. disc_rhs with the
    Q1 interpolants of nodal f and g).  A is symmetric (Sec. 4.1), so with w
    the solution of A w = dL/du on the DOFs, dL/df = M^T w and dL/dg = G^T w
    (F depends linearly on f and g).  Values of dL/du off the DOFs do not
    matter: u is 0 there whatever f and g are."""
    d = np.ravel(dLdu).astype(np.float64) * system.dof
    w = direct_solve(system, d)
    dLdg = system.G.T @ w
    if system.B is not None:
        # strong box values enter F as - B g
        dLdg = dLdg - system.B.T @ w
    return system.M.T @ w, dLdg


def adjoint_neumann(system: System, dLdu: np.ndarray):
    """dL/dg_N of the same loss with mixed boundary conditions: F also holds
    N g_N (Eq. disc_rhs), so dL/dg_N = N^T w with the w of ``adjoint``."""
    d = np.ravel(dLdu).astype(np.float64) * system.dof
    w = direct_solve(system, d)
    return system.Gn.T @ w

