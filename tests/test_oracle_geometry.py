"""Pins for the oracle's geometry (snapping, classes, cut polygons, quadrature).

Each test checks the oracle against something other than itself: hand values
from the definitions of Sec. 2 / Sec. 5.2, closed-form areas, pi r^2, exact
monomial integrals.
"""
import math

import numpy as np
import pytest

from oracle import ghostfem as gf
from paper_2505_05105_gb300 import workloads as wl


def test_snapping_rule():
    # Sec. 2: a point of Omega (psi < 0) with |psi| < h^alpha is snapped to 0
    h, alpha = 0.125, 1.75
    thr = h ** alpha
    psi = np.array([-2 * thr, -thr, -0.5 * thr, -1e-300, 0.0, 0.5 * thr, 3.0])
    out = gf.snap(psi, h, alpha)
    np.testing.assert_array_equal(out, [-2 * thr, -thr, 0.0, 0.0, 0.0, 0.5 * thr, 3.0])


def test_cell_classes_by_internal_vertex_count():
    # psi < 0 internal; psi = 0 external (Sec. 5.2 tie-break)
    psi = np.array([[-1.0, -1.0, 1.0],
                    [-1.0, -1.0, 0.0],
                    [0.0, 1.0, 1.0]])
    cls = gf.cell_classes(psi)
    # cell (ic, jc) uses psi[jc:jc+2, ic:ic+2]
    assert cls[0, 0] == gf.INTERNAL
    assert cls[0, 1] == gf.CUT        # two internal
    assert cls[1, 0] == gf.CUT        # two internal
    assert cls[1, 1] == gf.CUT        # one internal
    psi2 = np.ones((3, 3)); psi2[1, 1] = 0.0
    assert (gf.cell_classes(psi2) == gf.EXTERNAL).all()


@pytest.mark.parametrize("t1,t2", [(0.3, 0.7), (1.0, 1.0), (0.05, 0.9), (0.01, 0.5)])
def test_triangle_geometry(t1, t2):
    # internal v0; psi linear along the two legs gives theta = psi_in/(psi_in-psi_out)
    psi4 = np.array([-1.0, (1 - t1) / t1, (1 - t2) / t2, 7.0])
    cfg, pieces, th = gf.cut_pieces(psi4)
    assert cfg == "triangle"
    assert np.allclose(sorted(th), sorted([t1, t2]), rtol=1e-14)
    assert np.allclose(gf.triangle_legs(psi4), (t1, t2), rtol=1e-14)
    h = 0.01
    ints = gf.cell_integrals(pieces, 0.3, -0.2, h)
    assert ints.area == pytest.approx(0.5 * t1 * t2 * h * h, rel=1e-13)
    assert ints.length == pytest.approx(h * math.hypot(t1, t2), rel=1e-13)


@pytest.mark.parametrize("t1,t2", [(0.3, 0.7), (0.5, 0.5), (0.02, 0.9)])
def test_quad_and_pentagon_areas(t1, t2):
    h = 0.25
    # quad: v0, v1 internal; cut on the vertical edges at heights t1, t2
    psi4 = np.array([-t1, -t2, 1 - t1, 1 - t2])
    cfg, pieces, th = gf.cut_pieces(psi4)
    assert cfg == "quad"
    ints = gf.cell_integrals(pieces, 0.0, 0.0, h)
    assert ints.area == pytest.approx(0.5 * (t1 + t2) * h * h, rel=1e-13)
    assert ints.length == pytest.approx(h * math.hypot(1.0, t2 - t1), rel=1e-13)
    # pentagon: all but v3 internal; the removed corner has legs (1-s1), (1-s2)
    s1, s2 = t1, t2
    psi4 = np.array([-5.0, -s1, -s2, 1.0 - 0.0])
    # edges v1-v3 and v2-v3: theta = s/(s+1)
    a, b = s1 / (s1 + 1), s2 / (s2 + 1)
    cfg, pieces, th = gf.cut_pieces(psi4)
    assert cfg == "pentagon"
    ints = gf.cell_integrals(pieces, 0.0, 0.0, h)
    assert ints.area == pytest.approx(h * h * (1 - 0.5 * (1 - a) * (1 - b)), rel=1e-13)


def test_saddle_readings():
    # diagonal internal vertices: centre value decides hexagon vs two triangles
    cfg, pieces, _ = gf.cut_pieces(np.array([-1.0, 0.5, 0.5, -1.0]))   # mean < 0
    assert cfg == "hexagon" and len(pieces) == 1 and len(pieces[0].segments) == 2
    cfg, pieces, _ = gf.cut_pieces(np.array([-0.5, 1.0, 1.0, -0.5]))   # mean > 0
    assert cfg == "two_triangles" and len(pieces) == 2
    area = sum(gf.cell_integrals([p], 0, 0, 1.0).area for p in pieces)
    # each triangle has legs 1/3: area 2 * (1/3)^2 / 2
    assert area == pytest.approx(1.0 / 9.0, rel=1e-13)
    # hexagon = square minus two corner triangles with legs 2/3
    ints = gf.cell_integrals(gf.cut_pieces(np.array([-1.0, 0.5, 0.5, -1.0]))[1], 0, 0, 1.0)
    assert ints.area == pytest.approx(1 - 2 * 0.5 * (1 / 3) ** 2, rel=1e-13)


def test_zero_length_segment_dropped():
    # external vertex with psi = 0 (snapped): both intersection points coincide
    cfg, pieces, th = gf.cut_pieces(np.array([-1.0, -1.0, -1.0, 0.0]))
    assert cfg == "pentagon" and pieces[0].segments == []
    ints = gf.cell_integrals(pieces, 0, 0, 0.5)
    assert ints.area == pytest.approx(0.25, rel=1e-14)


@pytest.mark.parametrize("a,b", [(0, 0), (1, 0), (2, 1), (3, 1), (2, 2), (4, 0), (1, 3)])
def test_triangle_rule_exact_on_monomials(a, b):
    # int over the unit right triangle of x^a y^b = a! b! / (a+b+2)!
    X, W = gf.triangle_rule([0, 0], [1, 0], [0, 1])
    exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
    assert (W * X[:, 0] ** a * X[:, 1] ** b).sum() == pytest.approx(exact, rel=1e-13)


def test_segment_rule_exact():
    X, W = gf.segment_rule([0.0, 1.0], [2.0, 1.0])
    assert (W * X[:, 0] ** 5).sum() == pytest.approx(2 ** 6 / 6, rel=1e-13)


def test_active_area_and_perimeter_converge_to_disc():
    # area of Omega_h -> pi r^2 and |Gamma_h| -> 2 pi r, at second order
    r = 0.39
    errs, perr = [], []
    for N in (32, 64, 128):
        p = wl.circle64(N)
        s = gf.assemble_problem(p)
        area = (s.cls == gf.INTERNAL).sum() * p.h ** 2 + sum(c.ints.area for c in s.cut)
        per = sum(c.ints.length for c in s.cut)
        errs.append(abs(area - math.pi * r * r))
        perr.append(abs(per - 2 * math.pi * r))
    # snapping at h^1.75 perturbs at O(h^1.75); demand better than first order
    assert errs[2] < errs[0] / 6
    assert perr[2] < perr[0] / 6 and perr[2] < 1e-3


def test_config1_counts():
    # circle of radius 0.39 at (0.02, 0.01), 64 x 64 cells: DOFs and cut cells
    s = gf.assemble_problem(wl.circle64(64))
    assert int(s.dof.sum()) == 2157
    assert len(s.cut) == 200
