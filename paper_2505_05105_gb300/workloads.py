"""Seeded synthetic inputs: level sets, data and manufactured solutions.

This module only *defines problems*: a level-set function psi sampled at the
grid nodes, nodal source values f, nodal Dirichlet data g and, where one is
known, the manufactured solution.  It holds none of the ghost-FEM or multigrid
arithmetic, so both the CPU oracle and the CUDA path can take their inputs from
here without sharing any of the method's code.

Node layout: every array has shape (N+1, N+1) indexed [j, i] (y index first),
so ``a.ravel()`` gives the single node index k = i + j (N+1) of Sec. 5.1.
The domain is Omega = {psi < 0} (Sec. 2).

Problems
--------
* ``circle64``   - disc of radius 0.39 centred at (0.02, 0.01) in [-0.5, 0.5]^2,
  u = exp(x) sin(y) (harmonic, so f = 0), g = u.
* ``flower``     - r - 0.3 - 0.1 sin(5 atan2(y, x)) in [-0.5, 0.5]^2,
  u = sin(3x) cos(2y), f = 13 sin(3x) cos(2y), g = u.
* ``three_discs`` - union of three seeded discs minus a small disc, random
  Fourier f, g = 0 (the large multi-feature workload).
* ``batch_geometry`` - seeded ellipses / k-petal flowers of mixed sizes with a
  random Fourier f and g = 0.
* ``paper_circle``, ``paper_flower``, ``paper_hourglass`` - the level sets of
  the 2D experiments of Sec. 5.3 (homogeneous data; used for convergence
  factors).
* ``rectangle`` - the unit square cut by the vertical line psi = x - 1 +
  (1 - theta) h (Sec. 5.3): weak Dirichlet on the cut side, strong Dirichlet
  on the three sides of the box it touches (meta["box_strong"]).
* ``annulus``, ``leaf``, ``half_disc`` - mixed Dirichlet / Neumann problems:
  the annulus and leaf of Sec. 5.3 with a manufactured solution, and a disc
  cut by a straight Neumann side (patch tests).  They carry a per-cell
  ``neumann_mask`` (N, N) and nodal Neumann data ``gN`` (the outward normal
  derivative of u, the normal extended off the boundary from the level set
  that defines that part of it).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np


@dataclass
class Problem:
    name: str
    N: int
    x0: float
    y0: float
    h: float
    psi: np.ndarray
    f: np.ndarray
    g: np.ndarray
    u_exact: Optional[np.ndarray] = None
    meta: dict = field(default_factory=dict)
    neumann_mask: Optional[np.ndarray] = None   # (N, N) cells [jc, ic], uint8
    gN: Optional[np.ndarray] = None             # nodal Neumann data

    @property
    def shape(self):
        return (self.N + 1, self.N + 1)


def node_grid(N: int, x0: float, y0: float, h: float):
    """Nodal coordinates X[j, i] = x0 + i h, Y[j, i] = y0 + j h."""
    t = np.arange(N + 1, dtype=np.float64)
    X, Y = np.meshgrid(x0 + t * h, y0 + t * h, indexing="xy")
    return X, Y


def _unit_box(N):
    return -0.5, -0.5, 1.0 / N


def circle64(N: int = 64) -> Problem:
    x0, y0, h = _unit_box(N)
    X, Y = node_grid(N, x0, y0, h)
    psi = np.sqrt((X - 0.02) ** 2 + (Y - 0.01) ** 2) - 0.39
    u = np.exp(X) * np.sin(Y)
    return Problem("circle", N, x0, y0, h, psi, np.zeros_like(u), u.copy(), u)


def flower(N: int = 256, k: int = 5, phase: float = 0.0,
           r0: float = 0.3, amp: float = 0.1) -> Problem:
    x0, y0, h = _unit_box(N)
    X, Y = node_grid(N, x0, y0, h)
    r = np.sqrt(X * X + Y * Y)
    psi = r - r0 - amp * np.sin(k * np.arctan2(Y, X) + phase)
    u = np.sin(3 * X) * np.cos(2 * Y)
    f = 13.0 * np.sin(3 * X) * np.cos(2 * Y)
    return Problem("flower", N, x0, y0, h, psi, f, u.copy(), u,
                   meta={"k": k, "phase": phase})


def adjoint_target(p: Problem, seed: int) -> np.ndarray:
    """The adjoint workload's target u_t: the flower's manufactured solution
    sin 3x cos 2y with seeded phases (nodal, (N+1)^2)."""
    rng = np.random.default_rng(seed)
    a, b = rng.uniform(0, 2 * np.pi, 2)
    x, y = node_grid(p.N, p.x0, p.y0, p.h)
    return np.sin(3 * x + a) * np.cos(2 * y + b)


def fourier_source(X, Y, rng, modes: int = 8):
    """f = sum_m c_m sin(pi (p_m x + q_m y) + phi_m), c ~ N(0,1), p,q in 1..4."""
    c = rng.standard_normal(modes)
    p = rng.integers(1, 5, size=modes)
    q = rng.integers(1, 5, size=modes)
    ph = rng.uniform(0.0, 2.0 * np.pi, size=modes)
    f = np.zeros_like(X)
    for m in range(modes):
        f += c[m] * np.sin(np.pi * (p[m] * X + q[m] * Y) + ph[m])
    return f


def three_discs(N: int = 8192, seed: int = 0) -> Problem:
    """Union of three discs (radii U[0.1, 0.25]) minus a disc of radius 0.05
    centred on the first disc's centre; random 8-mode Fourier f; g = 0."""
    rng = np.random.default_rng(seed)
    r = rng.uniform(0.1, 0.25, size=3)
    c = np.stack([rng.uniform(-0.5 + ri + 0.02, 0.5 - ri - 0.02, size=2)
                  for ri in r])
    x0, y0, h = _unit_box(N)
    X, Y = node_grid(N, x0, y0, h)
    d = np.full_like(X, np.inf)
    for i in range(3):
        d = np.minimum(d, np.hypot(X - c[i, 0], Y - c[i, 1]) - r[i])
    psi = np.maximum(d, 0.05 - np.hypot(X - c[0, 0], Y - c[0, 1]))
    f = fourier_source(X, Y, rng)
    return Problem("three_discs", N, x0, y0, h, psi, f, np.zeros_like(f),
                   None, meta={"radii": r.tolist(), "centres": c.tolist(),
                               "seed": seed})


def batch_geometry(index: int, seed: int = 0, sizes=(64, 128, 256, 512)) -> Problem:
    """Member ``index`` of the seeded batch: an ellipse (semi-axes U[.15,.45],
    rotation U[0, pi]) or a k-petal flower (k in 3..7, random phase), grid size
    drawn from ``sizes``, random Fourier f and g = 0."""
    rng = np.random.default_rng([seed, index])
    N = int(rng.choice(sizes))
    x0, y0, h = _unit_box(N)
    X, Y = node_grid(N, x0, y0, h)
    if rng.uniform() < 0.5:
        a, b = rng.uniform(0.15, 0.45, size=2)
        rot = rng.uniform(0.0, np.pi)
        xr = np.cos(rot) * X + np.sin(rot) * Y
        yr = -np.sin(rot) * X + np.cos(rot) * Y
        psi = min(a, b) * (np.sqrt((xr / a) ** 2 + (yr / b) ** 2) - 1.0)
        meta = {"kind": "ellipse", "a": a, "b": b, "rot": rot}
    else:
        k = int(rng.integers(3, 8))
        ph = rng.uniform(0.0, 2.0 * np.pi)
        r = np.sqrt(X * X + Y * Y)
        psi = r - 0.3 - 0.1 * np.sin(k * np.arctan2(Y, X) + ph)
        meta = {"kind": "flower", "k": k, "phase": ph}
    f = fourier_source(X, Y, rng)
    return Problem(f"batch{index}", N, x0, y0, h, psi, f, np.zeros_like(f),
                   None, meta=meta)


# --- level sets of the paper's 2D experiments (Sec. 5.3), homogeneous data ---

def paper_circle(N: int) -> Problem:
    """psi = (x-0.5)^2 + (y-0.5)^2 - 0.4^2 on [0,1]^2."""
    h = 1.0 / N
    X, Y = node_grid(N, 0.0, 0.0, h)
    psi = (X - 0.5) ** 2 + (Y - 0.5) ** 2 - 0.16
    z = np.zeros_like(psi)
    return Problem("paper_circle", N, 0.0, 0.0, h, psi, z, z.copy())


def paper_flower(N: int) -> Problem:
    """Five-petal flower on [-1,1]^2."""
    h = 2.0 / N
    X, Y = node_grid(N, -1.0, -1.0, h)
    Xs = X - 0.03 * np.sqrt(3.0)
    Ys = Y - 0.04 * np.sqrt(2.0)
    R = np.sqrt(Xs ** 2 + Ys ** 2)
    psi = R - 0.52 - (Ys ** 5 + 5 * Xs ** 4 * Ys - 10 * Xs ** 2 * Ys ** 3) / (5 * R ** 5)
    z = np.zeros_like(psi)
    return Problem("paper_flower", N, -1.0, -1.0, h, psi, z, z.copy())


def paper_hourglass(N: int) -> Problem:
    """Quartic hourglass on [-1,1]^2."""
    h = 2.0 / N
    X, Y = node_grid(N, -1.0, -1.0, h)
    Xs = X - 0.03 * np.sqrt(3.0)
    Ys = Y - 0.04 * np.sqrt(2.0)
    psi = 256 * Ys ** 4 - 16 * Xs ** 4 - 128 * Ys ** 2 + 36 * Xs ** 2
    z = np.zeros_like(psi)
    return Problem("paper_hourglass", N, -1.0, -1.0, h, psi, z, z.copy())


def vertical_line(N: int, theta: float) -> Problem:
    """Half-plane x < 1 - (1-theta) h on [0,1]^2 shifted so that the domain is
    bounded away from the box; its cut cells are quads with both cut lengths
    theta h (the straight-cut rectangle of Sec. 5.3)."""
    h = 1.0 / N
    X, Y = node_grid(N, 0.0, 0.0, h)
    xc = 0.5 + theta * h
    psi = np.maximum(X - xc, np.maximum(0.25 - X, np.abs(Y - 0.5) - 0.3))
    z = np.zeros_like(psi)
    return Problem("vertical_line", N, 0.0, 0.0, h, psi, z, z.copy(),
                   meta={"theta": theta})


# --- mixed Dirichlet / Neumann problems ----------------------------------------

def cell_centres(N: int, x0: float, y0: float, h: float):
    """Cell centres Xc[jc, ic], Yc[jc, ic]."""
    t = np.arange(N, dtype=np.float64) + 0.5
    return np.meshgrid(x0 + t * h, y0 + t * h, indexing="xy")


def _sin3cos2(X, Y):
    u = np.sin(3 * X) * np.cos(2 * Y)
    ux = 3 * np.cos(3 * X) * np.cos(2 * Y)
    uy = -2 * np.sin(3 * X) * np.sin(2 * Y)
    return u, ux, uy, 13.0 * u


def annulus(N: int = 64, r1: float = 0.5, r2: float = 0.8) -> Problem:
    """Annulus r1 < r < r2 in [-1, 1]^2 (Sec. 5.3): Dirichlet on the inner
    circle, Neumann on the outer one; psi = max(r1^2 - r^2, r^2 - r2^2).
    u = sin 3x cos 2y, g_D = u, g_N = grad u . (x, y) / r.  A cut cell is
    Neumann when its centre lies outside the middle radius (r1 + r2) / 2."""
    h = 2.0 / N
    X, Y = node_grid(N, -1.0, -1.0, h)
    r2n = X * X + Y * Y
    psi = np.maximum(r1 * r1 - r2n, r2n - r2 * r2)
    u, ux, uy, f = _sin3cos2(X, Y)
    r = np.sqrt(r2n)
    gN = (ux * X + uy * Y) / np.where(r > 0, r, 1.0)
    Xc, Yc = cell_centres(N, -1.0, -1.0, h)
    mask = (np.hypot(Xc, Yc) > 0.5 * (r1 + r2)).astype(np.uint8)
    return Problem("annulus", N, -1.0, -1.0, h, psi, f, u.copy(), u,
                   meta={"r1": r1, "r2": r2}, neumann_mask=mask, gN=gN)


def leaf(N: int = 64) -> Problem:
    """Leaf of Sec. 5.3 in [-1, 1]^2: the intersection of two discs of radius
    0.7 centred at (-0.25 cos(pi/4), 0) and (0.25 sin(pi/4), 0), psi =
    max(R1 - 0.7, R2 - 0.7) (the paper prints R_1 twice; the second is read
    as R_2).  Dirichlet where x >= 0, Neumann where x < 0: a cut cell is
    Neumann when its centre has x < 0 and the second disc's level set is the
    larger one at all four of its corners, so that its boundary piece lies on
    that disc alone; the cells at the two corners of the leaf (on x = 0,
    where the discs meet) stay Dirichlet.  u = sin 3x cos 2y, g_N = grad u . n
    with n the unit radial direction of the disc whose level set is the
    larger at the node."""
    h = 2.0 / N
    X, Y = node_grid(N, -1.0, -1.0, h)
    xa, xb = -0.25 * np.cos(np.pi / 4), 0.25 * np.sin(np.pi / 4)
    R1, R2 = np.hypot(X - xa, Y), np.hypot(X - xb, Y)
    psi = np.maximum(R1 - 0.7, R2 - 0.7)
    u, ux, uy, f = _sin3cos2(X, Y)
    first = R1 - 0.7 >= R2 - 0.7
    cx = np.where(first, xa, xb)
    R = np.where(first, R1, R2)
    gN = (ux * (X - cx) + uy * Y) / np.where(R > 0, R, 1.0)
    Xc, _ = cell_centres(N, -1.0, -1.0, h)
    d2 = ~first
    on2 = d2[:-1, :-1] & d2[:-1, 1:] & d2[1:, :-1] & d2[1:, 1:]
    mask = ((Xc < 0.0) & on2).astype(np.uint8)
    return Problem("leaf", N, -1.0, -1.0, h, psi, f, u.copy(), u,
                   neumann_mask=mask, gN=gN)


def half_disc(N: int = 64, c: float = 0.1537) -> Problem:
    """The disc of circle64 cut by the straight side x = c: psi =
    max(|x - (0.02, 0.01)| - 0.39, x - c) in [-0.5, 0.5]^2.  A cut cell is
    Neumann when the straight side's term is the larger one at all four of
    its corners (its discrete boundary is then exactly on a vertical line,
    outward normal +x).  Data for u = exp(x) sin y: g_D = u, g_N = du/dx."""
    x0, y0, h = _unit_box(N)
    X, Y = node_grid(N, x0, y0, h)
    circ = np.sqrt((X - 0.02) ** 2 + (Y - 0.01) ** 2) - 0.39
    line = X - c
    psi = np.maximum(circ, line)
    u = np.exp(X) * np.sin(Y)
    ln = line >= circ
    mask = (ln[:-1, :-1] & ln[:-1, 1:] & ln[1:, :-1] & ln[1:, 1:]).astype(np.uint8)
    return Problem("half_disc", N, x0, y0, h, psi, np.zeros_like(u), u.copy(), u,
                   meta={"c": c}, neumann_mask=mask, gN=u.copy())


def rectangle(N: int = 128, theta: float = 0.5) -> Problem:
    """[0, 1]^2 cut by the vertical line x = 1 - (1 - theta) h (psi = x - 1 +
    (1 - theta) h, Sec. 5.3): every cut cell is a quadrilateral with cut
    sides theta h.  Weak (Nitsche) Dirichlet on the cut side, strong on the
    box sides x = 0, y = 0 and y = 1.  u = sin 3x cos 2y, f = 13 u, g = u at
    every node (the box nodes' strong values and the weak data)."""
    h = 1.0 / N
    X, Y = node_grid(N, 0.0, 0.0, h)
    psi = X - 1.0 + (1.0 - theta) * h
    u = np.sin(3 * X) * np.cos(2 * Y)
    return Problem("rectangle", N, 0.0, 0.0, h, psi, 13.0 * u, u.copy(), u,
                   meta={"theta": theta, "box_strong": True})

