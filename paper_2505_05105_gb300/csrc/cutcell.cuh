// Cut-cell geometry, exact quadrature and the local stabilisation constant,
// one thread per cut cell (setup path).
//
// Everything is computed in the reference square [0,1]^2 of the cell, where
// the 2D ghost-FEM element matrices are independent of h:
//   Ke = S + (lambda h) Ms - Bn - Bn^T       (Eq. disc_bil_form on K)
//   Gk = (lambda h) Ms - Bn^T                 (Eq. disc_rhs boundary load)
//   Mk = h^2 Mref                             (mass of K cap Omega_h)
// and for a cell whose boundary piece is Neumann (no boundary terms in
// Eq. disc_bil_form; the load int g_N phi_i in Eq. disc_rhs):
//   Ke = S,  Gk = 0,  Nk = h Ms
// with S_ij = int_P grad phi_i . grad phi_j, Mref_ij = int_P phi_i phi_j over
// the cut polygon P, and on the boundary segments (reference length, outward
// normal n) Ms_ij = int phi_i phi_j, Bn_ij = int (n . grad phi_j) phi_i.
//
// Cut configurations follow Sec. 5.2: the vertex signs give a triangle (1
// internal vertex), quadrilateral (2 adjacent), pentagon (3); the cut points
// sit at theta = psi_in / (psi_in - psi_out) along sign-changing edges.  Two
// internal vertices on a diagonal (not covered by the paper) are resolved by
// the bilinear centre value: mean(psi) < 0 -> hexagon, else two triangles.
//
// C(K) h (Sec. 5.2): triangles use Eq. c_triangle, pentagons and hexagons use
// Eq. c_pentagon (3 sqrt 2), quadrilaterals and two-triangle cells use the
// definition: the largest eigenvalue of the local pencil (K, M) restricted to
// a complement of the constants (Sec. 4.4's rank-based definition), solved
// here in the basis {x - a, y - b, (x - a)(y - b)/d} centred on the polygon
// so that M stays well conditioned for small cuts.
#pragma once

#include <math.h>

namespace cutcell {

enum Config : int { CFG_EXT = 0, CFG_INT = 1, CFG_TRI = 2, CFG_QUAD = 3, CFG_PENT = 4,
                    CFG_HEX = 5, CFG_TWO_TRI = 6 };

struct Geom {
  int config;
  int npiece;
  int npt[2];
  double px[2][6], py[2][6];      // polygons, counter-clockwise
  int nseg;
  double ax[2], ay[2], bx[2], by[2];   // segments a -> b (outward normal on the right)
  double th[2];                   // triangle legs
};

// 3-point Gauss-Legendre on [0, 1]
__device__ __forceinline__ void gl3(double* s, double* w) {
  const double r = 0.38729833462074168852;   // sqrt(3/5) / 2
  s[0] = 0.5 - r; s[1] = 0.5; s[2] = 0.5 + r;
  w[0] = 5.0 / 18.0; w[1] = 8.0 / 18.0; w[2] = 5.0 / 18.0;
}

__device__ inline void build_geometry(const double psi[4], Geom& g) {
  // local vertices v0 (0,0), v1 (1,0), v2 (0,1), v3 (1,1); walk v0 v1 v3 v2
  const int ccw[4] = {0, 1, 3, 2};
  const double vx[4] = {0.0, 1.0, 0.0, 1.0};
  const double vy[4] = {0.0, 0.0, 1.0, 1.0};
  bool in[4];
  int nin = 0;
  for (int v = 0; v < 4; ++v) { in[v] = psi[v] < 0.0; nin += in[v]; }
  g.npiece = 0; g.nseg = 0; g.th[0] = g.th[1] = 0.0;
  if (nin == 0) { g.config = CFG_EXT; return; }
  if (nin == 4) {
    g.config = CFG_INT; g.npiece = 1; g.npt[0] = 4;
    for (int e = 0; e < 4; ++e) { g.px[0][e] = vx[ccw[e]]; g.py[0][e] = vy[ccw[e]]; }
    return;
  }
  double x[6], y[6];
  int kind[6];        // 0 vertex, 1 exit, 2 entry
  int m = 0;
  for (int e = 0; e < 4; ++e) {
    int a = ccw[e], b = ccw[(e + 1) & 3];
    if (in[a]) { x[m] = vx[a]; y[m] = vy[a]; kind[m] = 0; ++m; }
    if (in[a] != in[b]) {
      int ii = in[a] ? a : b, io = in[a] ? b : a;
      double t = psi[ii] / (psi[ii] - psi[io]);
      x[m] = vx[ii] + t * (vx[io] - vx[ii]);
      y[m] = vy[ii] + t * (vy[io] - vy[ii]);
      kind[m] = in[a] ? 1 : 2;
      ++m;
    }
  }
  bool diag = (nin == 2) && (in[0] == in[3]);
  bool two = false;
  if (diag) {
    double mean = (psi[0] + psi[1] + psi[2] + psi[3]) * 0.25;
    two = !(mean < 0.0);
  }
  if (!two) {
    g.config = diag ? CFG_HEX : (nin == 1 ? CFG_TRI : (nin == 2 ? CFG_QUAD : CFG_PENT));
    g.npiece = 1; g.npt[0] = m;
    for (int k = 0; k < m; ++k) { g.px[0][k] = x[k]; g.py[0][k] = y[k]; }
    for (int k = 0; k < m; ++k) {
      int q = (k + 1) % m;
      if (kind[k] == 1 && kind[q] == 2 && !(x[k] == x[q] && y[k] == y[q])) {
        g.ax[g.nseg] = x[k]; g.ay[g.nseg] = y[k];
        g.bx[g.nseg] = x[q]; g.by[g.nseg] = y[q];
        ++g.nseg;
      }
    }
    if (nin == 1) {
      // legs at the internal vertex along its two edges
      int v = in[0] ? 0 : (in[1] ? 1 : (in[2] ? 2 : 3));
      int w0 = (v == 0 || v == 3) ? 1 : 0;
      int w1 = (v == 0 || v == 3) ? 2 : 3;
      g.th[0] = psi[v] / (psi[v] - psi[w0]);
      g.th[1] = psi[v] / (psi[v] - psi[w1]);
    }
    return;
  }
  // two triangles: (entry, vertex, exit) around each internal vertex
  g.config = CFG_TWO_TRI;
  for (int k = 0; k < m; ++k) {
    if (kind[k] != 0) continue;
    int pm = (k + m - 1) % m, pp = (k + 1) % m;
    int P = g.npiece++;
    g.npt[P] = 3;
    g.px[P][0] = x[pm]; g.py[P][0] = y[pm];
    g.px[P][1] = x[k];  g.py[P][1] = y[k];
    g.px[P][2] = x[pp]; g.py[P][2] = y[pp];
    if (!(x[pp] == x[pm] && y[pp] == y[pm])) {
      g.ax[g.nseg] = x[pp]; g.ay[g.nseg] = y[pp];
      g.bx[g.nseg] = x[pm]; g.by[g.nseg] = y[pm];
      ++g.nseg;
    }
  }
}

__device__ __forceinline__ void q1(double xi, double et, double phi[4], double gx[4], double gy[4]) {
  phi[0] = (1.0 - xi) * (1.0 - et); phi[1] = xi * (1.0 - et);
  phi[2] = (1.0 - xi) * et;         phi[3] = xi * et;
  gx[0] = -(1.0 - et); gx[1] = 1.0 - et; gx[2] = -et;        gx[3] = et;
  gy[0] = -(1.0 - xi); gy[1] = -xi;      gy[2] = 1.0 - xi;   gy[3] = xi;
}

// Largest eigenvalue of a symmetric 3x3 matrix by cyclic Jacobi rotations.
__device__ inline double sym3_max_eig(double A[3][3]) {
  for (int sweep = 0; sweep < 30; ++sweep) {
    double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    double dn = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
    if (off <= 1e-34 * dn || off == 0.0) break;
    for (int p = 0; p < 2; ++p) {
      for (int q = p + 1; q < 3; ++q) {
        double apq = A[p][q];
        if (apq == 0.0) continue;
        double tau = (A[q][q] - A[p][p]) / (2.0 * apq);
        double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        // A <- J^T A J, rotation in the (p, q) plane
        for (int k = 0; k < 3; ++k) {
          double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < 3; ++k) {
          double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
        }
        A[p][q] = A[q][p] = 0.0;
      }
    }
  }
  return fmax(A[0][0], fmax(A[1][1], A[2][2]));
}

// Largest generalized eigenvalue of (K, M), M SPD 3x3: Cholesky M = L L^T,
// B = L^{-1} K L^{-T}, largest eigenvalue of B.
__device__ inline double gen3_max_eig(const double K[3][3], const double M[3][3]) {
  double L[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int j = 0; j < 3; ++j) {
    double d = M[j][j];
    for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
    if (!(d > 0.0)) return 0.0;
    L[j][j] = sqrt(d);
    for (int i = j + 1; i < 3; ++i) {
      double s = M[i][j];
      for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
      L[i][j] = s / L[j][j];
    }
  }
  // X = L^{-1} K  (forward substitution on each column)
  double X[3][3];
  for (int c = 0; c < 3; ++c) {
    for (int i = 0; i < 3; ++i) {
      double s = K[i][c];
      for (int k = 0; k < i; ++k) s -= L[i][k] * X[k][c];
      X[i][c] = s / L[i][i];
    }
  }
  // B = X L^{-T}: B^T = L^{-1} X^T
  double B[3][3];
  for (int r = 0; r < 3; ++r) {
    for (int i = 0; i < 3; ++i) {
      double s = X[r][i];
      for (int k = 0; k < i; ++k) s -= L[i][k] * B[r][k];
      B[r][i] = s / L[i][i];
    }
  }
  for (int i = 0; i < 3; ++i)
    for (int j = i + 1; j < 3; ++j) {
      double v = 0.5 * (B[i][j] + B[j][i]);
      B[i][j] = B[j][i] = v;
    }
  return sym3_max_eig(B);
}

// Eq. c_triangle times h, legs t1 h and t2 h.
__device__ inline double c_triangle_h(double t1, double t2) {
  double a2 = t1 * t1, b2 = t2 * t2;
  double a4 = a2 * a2, b4 = b2 * b2;
  double s = a2 + b2;
  double num = sqrt(s / a2) * (3.0 * a4 + 3.0 * b4 + sqrt(3.0 * (a4 * a4 + 10.0 * a4 * b4 + b4 * b4)));
  return num / (t2 * s * s);
}

struct CellOut {
  double Ke[16], Gk[16], Mk[16], Nk[16];
  double S[16];    // volume stiffness on K cap Omega_h (h-independent in 2D)
  double Kn[16];   // int_{Gamma_h cap K} (n . grad phi_i)(n . grad phi_j), times h
  double C, lam;
  double area, length;
  int config;
};

// Element matrices of one cut cell.  psi: corner values v0..v3 (snapped).
// ch_global >= 0: lambda h = gamma ch_global on this cell (the global
// constant of Sec. 5.2 times h) instead of the local gamma C(K) h.
__device__ inline void cut_cell_matrices(const double psi[4], double h, double gamma, CellOut& o,
                                         bool neumann = false, double ch_global = -1.0) {
  Geom g;
  build_geometry(psi, g);
  o.config = g.config;
  double S[4][4] = {}, Mr[4][4] = {}, Ms[4][4] = {}, Bn[4][4] = {}, Kn[4][4] = {};
  double M3[3][3] = {}, K3[3][3] = {};
  double gs[3], gw[3];
  gl3(gs, gw);
  // centre and scale of the basis of the complement of constants
  double ca = 0.0, cb = 0.0, xmin = 1.0, xmax = 0.0, ymin = 1.0, ymax = 0.0;
  int ncount = 0;
  for (int P = 0; P < g.npiece; ++P)
    for (int k = 0; k < g.npt[P]; ++k) {
      ca += g.px[P][k]; cb += g.py[P][k]; ++ncount;
      xmin = fmin(xmin, g.px[P][k]); xmax = fmax(xmax, g.px[P][k]);
      ymin = fmin(ymin, g.py[P][k]); ymax = fmax(ymax, g.py[P][k]);
    }
  if (ncount) { ca /= ncount; cb /= ncount; }
  double d = fmax(fmax(xmax - xmin, ymax - ymin), 1e-300);
  double area = 0.0, length = 0.0;
  for (int P = 0; P < g.npiece; ++P) {
    for (int k = 1; k + 1 < g.npt[P]; ++k) {
      double Ax = g.px[P][0], Ay = g.py[P][0];
      double Bx = g.px[P][k] - Ax, By = g.py[P][k] - Ay;
      double Cx = g.px[P][k + 1] - Ax, Cy = g.py[P][k + 1] - Ay;
      double jac = fabs(Bx * Cy - By * Cx);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          double s = gs[a], t = gs[b];
          double w = jac * s * gw[a] * gw[b];
          double xi = Ax + s * (1.0 - t) * Bx + s * t * Cx;
          double et = Ay + s * (1.0 - t) * By + s * t * Cy;
          double phi[4], gx[4], gy[4];
          q1(xi, et, phi, gx, gy);
          for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) {
              S[i][j] += w * (gx[i] * gx[j] + gy[i] * gy[j]);
              Mr[i][j] += w * phi[i] * phi[j];
            }
          double bx[3] = {1.0, 0.0, (et - cb) / d};
          double by[3] = {0.0, 1.0, (xi - ca) / d};
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) M3[i][j] += w * (bx[i] * bx[j] + by[i] * by[j]);
          area += w;
        }
    }
  }
  for (int e = 0; e < g.nseg; ++e) {
    double dx = g.bx[e] - g.ax[e], dy = g.by[e] - g.ay[e];
    double len = sqrt(dx * dx + dy * dy);
    double nx = dy / len, ny = -dx / len;
    length += len;
    for (int a = 0; a < 3; ++a) {
      double w = len * gw[a];
      double xi = g.ax[e] + gs[a] * dx, et = g.ay[e] + gs[a] * dy;
      double phi[4], gx[4], gy[4];
      q1(xi, et, phi, gx, gy);
      double dn[4];
      for (int i = 0; i < 4; ++i) dn[i] = nx * gx[i] + ny * gy[i];
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
          Ms[i][j] += w * phi[i] * phi[j];
          Bn[i][j] += w * dn[j] * phi[i];
          Kn[i][j] += w * dn[i] * dn[j];
        }
      double gb[3] = {nx, ny, (nx * (et - cb) + ny * (xi - ca)) / d};
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) K3[i][j] += w * gb[i] * gb[j];
    }
  }
  double Ch;
  if (g.config == CFG_TRI) Ch = c_triangle_h(g.th[0], g.th[1]);
  else if (g.config == CFG_PENT || g.config == CFG_HEX) Ch = 3.0 * sqrt(2.0);
  else if (length > 0.0) Ch = gen3_max_eig(K3, M3);
  else Ch = 0.0;
  double lamh = gamma * (ch_global >= 0.0 ? ch_global : Ch);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      if (neumann) {
        o.Ke[i * 4 + j] = S[i][j];
        o.Gk[i * 4 + j] = 0.0;
        o.Nk[i * 4 + j] = h * Ms[i][j];
      } else {
        o.Ke[i * 4 + j] = S[i][j] + lamh * Ms[i][j] - Bn[i][j] - Bn[j][i];
        o.Gk[i * 4 + j] = lamh * Ms[i][j] - Bn[j][i];
        o.Nk[i * 4 + j] = 0.0;
      }
      o.Mk[i * 4 + j] = h * h * Mr[i][j];
      o.S[i * 4 + j] = S[i][j];
      o.Kn[i * 4 + j] = neumann ? 0.0 : Kn[i][j];
    }
  // exact symmetry of Ke (the two halves are summed in different orders)
  for (int i = 0; i < 4; ++i)
    for (int j = i + 1; j < 4; ++j) {
      double v = 0.5 * (o.Ke[i * 4 + j] + o.Ke[j * 4 + i]);
      o.Ke[i * 4 + j] = o.Ke[j * 4 + i] = v;
    }
  o.C = Ch / h;
  o.lam = lamh / h;
  o.area = area * h * h;
  o.length = length * h;
}

}  // namespace cutcell
