// tables.cpp -- reference-element data of the device path: orthonormal Dubiner basis
// (Eq. dubiner) at the area and edge quadrature points, the quadrature rules and the
// vertex-to-linear-mode map.
//
// The Dubiner functions phi_ij = sqrt((2i+1)(i+j+1)/2) P_i(a) ((1-b)/2)^i P_j^{(2i+1,0)}(b),
// collapsed coordinates a = 2(1+r)/(1-s) - 1, b = s on the reference triangle
// (-1,-1),(1,-1),(-1,1), are evaluated here from the explicit sum formulas
//   P_n^{(al,0)}(x) = sum_k C(n+al, n-k) C(n, k) ((x-1)/2)^k ((x+1)/2)^{n-k},
//   P_i(a) ((1-s)/2)^i = 2^{-i} sum_k C(i,k)^2 (r+s)^k (1+r)^{i-k},
// which are polynomials in (r, s) with no singular point.  Ordering: total degree i+j, then j.
//
// Quadrature: area rules exact to degree 2p+1 with positive weights and full triangle symmetry
// (p=1: centroid 27/60, edge midpoints 8/60, vertices 3/60 of the area -- Stroud's degree-3
// rule; p=2: Radon's 7-point degree-5 rule, centroid 9/40, orbits a = (6 -/+ sqrt 15)/21 with
// weights (155 -/+ sqrt 15)/1200); edges: Gauss-Legendre with p+1 points.
#include <cmath>
#include <cstddef>
#include <cstring>

#include "layout.h"

namespace dg {

static double binom(double n, int k) {
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r *= (n - k + i) / i;
  return r;
}

static double ipow(double x, int n) {
  double r = 1.0;
  for (int i = 0; i < n; ++i) r *= x;
  return r;
}

// value and derivative of P_n^{(al,0)}(x)
static void jacobi(int n, double al, double x, double& v, double& dv) {
  v = 0.0;
  dv = 0.0;
  const double a = 0.5 * (x - 1.0), b = 0.5 * (x + 1.0);
  for (int k = 0; k <= n; ++k) {
    const double c = binom(n + al, n - k) * binom(n, k);
    v += c * ipow(a, k) * ipow(b, n - k);
    if (k > 0) dv += c * 0.5 * k * ipow(a, k - 1) * ipow(b, n - k);
    if (n - k > 0) dv += c * 0.5 * (n - k) * ipow(a, k) * ipow(b, n - k - 1);
  }
}

// value and (r, s) derivatives of P_i(a) ((1-s)/2)^i
static void collapsed_legendre(int i, double r, double s, double& v, double& dr, double& ds) {
  v = dr = ds = 0.0;
  const double u = r + s, w = 1.0 + r, sc = std::ldexp(1.0, -i);
  for (int k = 0; k <= i; ++k) {
    const double c = sc * binom(i, k) * binom(i, k);
    v += c * ipow(u, k) * ipow(w, i - k);
    double du = (k > 0) ? k * ipow(u, k - 1) * ipow(w, i - k) : 0.0;   // d/du
    double dw = (i - k > 0) ? (i - k) * ipow(u, k) * ipow(w, i - k - 1) : 0.0;  // d/dw
    dr += c * (du + dw);  // u and w both depend on r with unit slope
    ds += c * du;
  }
}

void dubiner_eval(int p, double r, double s, double* phi, double* dphr, double* dphs) {
  int m = 0;
  for (int d = 0; d <= p; ++d)
    for (int j = 0; j <= d; ++j) {
      const int i = d - j;
      double q, qr, qs, pj, dpj;
      collapsed_legendre(i, r, s, q, qr, qs);
      jacobi(j, 2.0 * i + 1.0, s, pj, dpj);
      const double c = std::sqrt((2.0 * i + 1.0) * (i + j + 1.0) / 2.0);
      phi[m] = c * q * pj;
      if (dphr) dphr[m] = c * qr * pj;
      if (dphs) dphs[m] = c * (qs * pj + q * dpj);
      ++m;
    }
}

static void rs_of(const double l[3], double& r, double& s) {
  // (r, s) = l0 (-1,-1) + l1 (1,-1) + l2 (-1,1)
  r = -l[0] + l[1] - l[2];
  s = -l[0] - l[1] + l[2];
}

void build_tables(int p, RefTab<double>& t) {
  std::memset(&t, 0, sizeof t);
  t.np = (p + 1) * (p + 2) / 2;
  // area rule (barycentric points, weights as fractions of the area)
  double L[MAXNQ][3], W[MAXNQ];
  int n = 0;
  auto orbit = [&](double a, double w) {  // (1-2a, a, a) and its rotations
    for (int k = 0; k < 3; ++k) {
      L[n][k] = 1.0 - 2.0 * a;
      L[n][(k + 1) % 3] = a;
      L[n][(k + 2) % 3] = a;
      W[n++] = w;
    }
  };
  L[0][0] = L[0][1] = L[0][2] = 1.0 / 3.0;
  if (p <= 0) {
    W[0] = 1.0;
    n = 1;
  } else if (p == 1) {
    W[n++] = 27.0 / 60.0;
    orbit(0.5, 8.0 / 60.0);   // (0, 1/2, 1/2): edge midpoints
    orbit(0.0, 3.0 / 60.0);   // (1, 0, 0): vertices
  } else {
    W[n++] = 9.0 / 40.0;
    const double r15 = std::sqrt(15.0);
    orbit((6.0 - r15) / 21.0, (155.0 - r15) / 1200.0);
    orbit((6.0 + r15) / 21.0, (155.0 + r15) / 1200.0);
  }
  t.nq = n;
  for (int q = 0; q < n; ++q) {
    double r, s;
    rs_of(L[q], r, s);
    t.qw[q] = 2.0 * W[q];
    for (int k = 0; k < 3; ++k) t.ql[q][k] = L[q][k];
    dubiner_eval(p, r, s, t.qphi[q], t.qdr[q], t.qds[q]);
  }
  // Gauss-Legendre on [-1, 1]
  t.ng = p + 1;
  double xi[MAXNG], gw[MAXNG];
  if (p <= 0) {
    xi[0] = 0.0; gw[0] = 2.0;
  } else if (p == 1) {
    xi[0] = -1.0 / std::sqrt(3.0); xi[1] = -xi[0]; gw[0] = gw[1] = 1.0;
  } else {
    xi[0] = -std::sqrt(0.6); xi[1] = 0.0; xi[2] = -xi[0];
    gw[0] = gw[2] = 5.0 / 9.0; gw[1] = 8.0 / 9.0;
  }
  for (int k = 0; k < t.ng; ++k) t.gw[k] = gw[k];
  for (int j = 0; j < 3; ++j)
    for (int k = 0; k < t.ng; ++k) {
      double l[3] = {0, 0, 0}, r, s;
      l[j] = 0.5 * (1.0 - xi[k]);
      l[(j + 1) % 3] = 0.5 * (1.0 + xi[k]);
      for (int c = 0; c < 3; ++c) t.el[j][k][c] = l[c];
      rs_of(l, r, s);
      dubiner_eval(p, r, s, t.ephi[j][k], nullptr, nullptr);
    }
  // vertices, and the map from vertex values of a linear function to its modes 1 and 2
  double V[3][3];
  for (int i = 0; i < 3; ++i) {
    double l[3] = {0, 0, 0}, r, s;
    l[i] = 1.0;
    rs_of(l, r, s);
    dubiner_eval(p, r, s, t.vphi[i], nullptr, nullptr);
    double lin[MAXNP];
    dubiner_eval(1, r, s, lin, nullptr, nullptr);
    for (int m = 0; m < 3; ++m) V[i][m] = lin[m];
  }
  // invert V (rows: vertices, columns: linear modes) by Cramer's rule
  const double det = V[0][0] * (V[1][1] * V[2][2] - V[1][2] * V[2][1]) - V[0][1] * (V[1][0] * V[2][2] - V[1][2] * V[2][0]) +
                     V[0][2] * (V[1][0] * V[2][1] - V[1][1] * V[2][0]);
  double inv[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      const int r1 = (r + 1) % 3, r2 = (r + 2) % 3, c1 = (c + 1) % 3, c2 = (c + 2) % 3;
      inv[c][r] = (V[r1][c1] * V[r2][c2] - V[r1][c2] * V[r2][c1]) / det;
    }
  for (int m = 0; m < 2; ++m)
    for (int i = 0; i < 3; ++i) t.vinv[m][i] = inv[m + 1][i];
  // edge midpoints (edge j joins vertices j and j+1)
  for (int j = 0; j < 3; ++j) {
    double l[3] = {0, 0, 0}, r, s;
    l[j] = 0.5;
    l[(j + 1) % 3] = 0.5;
    rs_of(l, r, s);
    dubiner_eval(p, r, s, t.mphi[j], nullptr, nullptr);
  }
  t.phi0 = 1.0 / std::sqrt(2.0);
  for (int q = 0; q < t.nq; ++q) t.qwT[q] = t.qw[q];
  for (int m = 0; m < t.np; ++m)
    for (int i = 0; i < 3; ++i) t.vabs[m] = std::max(t.vabs[m], std::fabs(t.vphi[i][m]));
  for (int m = 0; m < t.np; ++m)
    for (int q = 0; q < t.nq; ++q) {
      t.qphiT[m][q] = t.qphi[q][m];
      t.qwphiT[m][q] = t.qw[q] * t.qphi[q][m];
      t.qdrT[m][q] = t.qdr[q][m];
      t.qdsT[m][q] = t.qds[q][m];
    }
}

void tables_to_float(const RefTab<double>& d, RefTab<float>& f) {
  std::memset(&f, 0, sizeof f);
  f.nq = d.nq; f.ng = d.ng; f.np = d.np;
  const double* src = &d.qw[0];
  float* dst = &f.qw[0];
  const size_t n = (sizeof(RefTab<double>) - offsetof(RefTab<double>, qw)) / sizeof(double);
  for (size_t i = 0; i < n; ++i) dst[i] = (float)src[i];
}

}  // namespace dg
