// tables.cpp -- 1-D band tables of the Q2-Q1 element matrices (host, FP64).
//
// On the uniform tensor-product grid every operator of Sec. 2.2 factors
// into 1-D element integrals; they are assembled here into per-node bands
// (offsets -2..2 on the Q2 node line, -1..1 on the Q1 node line) by 3-point
// Gauss quadrature on each element (exact: the integrands have degree <= 5).
//   M1_ik = int phi_i phi_k         K1_ik = int phi_i' phi_k'
//   W1_ik = int phi_i (1 - s^2) phi_k'   X1_ik = int phi_i s phi_k
//   G1_ki = int psi_k phi_i'         H1_ki = int psi_k phi_i  (Q1 row k, Q2 column i)
#include <cmath>
#include <vector>

#include "tables.h"

namespace pint {

namespace {

void gauss3(double xi[3], double w[3]) {
  const double a = std::sqrt(0.6) / 2.0;
  xi[0] = 0.5 - a;
  xi[1] = 0.5;
  xi[2] = 0.5 + a;
  w[0] = 5.0 / 18.0;
  w[1] = 8.0 / 18.0;
  w[2] = 5.0 / 18.0;
}

// quadratic Lagrange basis on [0, 1] with nodes 0, 1/2, 1 (value, d/dxi)
void quad_basis(double t, double v[3], double d[3]) {
  v[0] = 2.0 * (t - 0.5) * (t - 1.0);
  v[1] = -4.0 * t * (t - 1.0);
  v[2] = 2.0 * t * (t - 0.5);
  d[0] = 4.0 * t - 3.0;
  d[1] = 4.0 - 8.0 * t;
  d[2] = 4.0 * t - 1.0;
}
void lin_basis(double t, double v[2], double d[2]) {
  v[0] = 1.0 - t;
  v[1] = t;
  d[0] = -1.0;
  d[1] = 1.0;
}

// 4-point Gauss-Legendre rule mapped to [0, 1]: nodes (1 -+ sqrt(3/7 +- 2/7
// sqrt(6/5))) / 2, weights (18 -+ sqrt(30)) / 72.
void gauss4(double xi[4], double w[4]) {
  const double a = std::sqrt(3.0 / 7.0 - 2.0 / 7.0 * std::sqrt(6.0 / 5.0));
  const double b = std::sqrt(3.0 / 7.0 + 2.0 / 7.0 * std::sqrt(6.0 / 5.0));
  const double wa = (18.0 + std::sqrt(30.0)) / 72.0, wb = (18.0 - std::sqrt(30.0)) / 72.0;
  xi[0] = 0.5 * (1.0 - b);
  xi[1] = 0.5 * (1.0 - a);
  xi[2] = 0.5 * (1.0 + a);
  xi[3] = 0.5 * (1.0 + b);
  w[0] = wb;
  w[1] = wa;
  w[2] = wa;
  w[3] = wb;
}

// Sec. 5.2 wind: c1 (A^2 y, -B^2 (x - 1/2)) inside the ellipse c1 >= 0 about
// (1/2, 0), c2 (-A^2 y, B^2 (x + 1/2)) inside c2 >= 0 about (-1/2, 0), else 0,
// with c = 1 - sqrt((B (x -+ 1/2))^2 + (A y)^2), A = 100/99, B = 100/49.
void two_vortex(double x, double y, double& wx, double& wy) {
  const double A = 100.0 / 99.0, B = 100.0 / 49.0;
  const double c1 = 1.0 - std::sqrt((B * (x - 0.5)) * (B * (x - 0.5)) + (A * y) * (A * y));
  const double c2 = 1.0 - std::sqrt((B * (x + 0.5)) * (B * (x + 0.5)) + (A * y) * (A * y));
  if (c1 >= 0.0) {
    wx = c1 * A * A * y;
    wy = -c1 * B * B * (x - 0.5);
  } else if (c2 >= 0.0) {
    wx = -c2 * A * A * y;
    wy = c2 * B * B * (x + 0.5);
  } else {
    wx = wy = 0.0;
  }
}

// Wind at Gauss point (qa, qb) of element (ex, ey): the two-vortex formula
// (wind == nullptr), or the Q2 interpolant of nodal values wind[2][(2N+1)^2].
void wind_at(int N, double x0, double h, const double* wind, int ex, int ey, const double xi[4], int qa, int qb,
             double& wx, double& wy) {
  if (!wind) {
    two_vortex(x0 + (ex + xi[qa]) * h, x0 + (ey + xi[qb]) * h, wx, wy);
    return;
  }
  const int n2 = 2 * N + 1;
  double va[3], vb[3], d[3];
  quad_basis(xi[qa], va, d);
  quad_basis(xi[qb], vb, d);
  wx = wy = 0.0;
  for (int b = 0; b < 3; ++b)
    for (int a = 0; a < 3; ++a) {
      const size_t node = (size_t)(2 * ey + b) * n2 + (2 * ex + a);
      wx += va[a] * vb[b] * wind[node];
      wy += va[a] * vb[b] * wind[(size_t)n2 * n2 + node];
    }
}

// Raw convection stencils int phi_i (w . grad phi_j) of one element family
// (p nodes per element side: 3 for Q2, 2 for Q1; band half-width p - 1),
// then the skew part.  Node (ix, iy) of an n x n grid, n = (p - 1) N + 1.
void convection_stencils(int N, double x0, double x1, int p, const double* wind, std::vector<double>& out) {
  const int n = (p - 1) * N + 1, hw = p - 1, bw = 2 * hw + 1, nk = bw * bw;
  const double h = (x1 - x0) / N;
  double xi[4], wq[4];
  gauss4(xi, wq);
  std::vector<double> raw((size_t)n * n * nk, 0.0);
  double v[4][3], d[4][3];
  for (int q = 0; q < 4; ++q) {
    double vv[3], dd[3];
    if (p == 3)
      quad_basis(xi[q], vv, dd);
    else
      lin_basis(xi[q], vv, dd);
    for (int a = 0; a < p; ++a) {
      v[q][a] = vv[a];
      d[q][a] = dd[a] / h;
    }
  }
  for (int ey = 0; ey < N; ++ey)
    for (int ex = 0; ex < N; ++ex)
      for (int qb = 0; qb < 4; ++qb)
        for (int qa = 0; qa < 4; ++qa) {
          double wx, wy;
          wind_at(N, x0, h, wind, ex, ey, xi, qa, qb, wx, wy);
          const double W = wq[qa] * wq[qb] * h * h;
          for (int bi = 0; bi < p; ++bi)
            for (int ai = 0; ai < p; ++ai) {
              const double phi = v[qa][ai] * v[qb][bi];
              const int ix = hw * ex + ai, iy = hw * ey + bi;
              double* row = raw.data() + ((size_t)iy * n + ix) * nk;
              for (int bj = 0; bj < p; ++bj)
                for (int aj = 0; aj < p; ++aj) {
                  const double g = wx * d[qa][aj] * v[qb][bj] + wy * v[qa][aj] * d[qb][bj];
                  row[(bj - bi + hw) * bw + (aj - ai + hw)] += W * phi * g;
                }
            }
        }
  out.assign(raw.size(), 0.0);
  for (int iy = 0; iy < n; ++iy)
    for (int ix = 0; ix < n; ++ix)
      for (int dy = -hw; dy <= hw; ++dy)
        for (int dx = -hw; dx <= hw; ++dx) {
          const int jx = ix + dx, jy = iy + dy;
          if (jx < 0 || jx >= n || jy < 0 || jy >= n) continue;
          const double nij = raw[((size_t)iy * n + ix) * nk + (dy + hw) * bw + (dx + hw)];
          const double nji = raw[((size_t)jy * n + jx) * nk + (-dy + hw) * bw + (-dx + hw)];
          out[((size_t)iy * n + ix) * nk + (dy + hw) * bw + (dx + hw)] = 0.5 * (nij - nji);
        }
}

}  // namespace

void build_two_vortex_stencils(int N, double x0, double x1, std::vector<double>& q2, std::vector<double>& q1) {
  convection_stencils(N, x0, x1, 3, nullptr, q2);
  convection_stencils(N, x0, x1, 2, nullptr, q1);
}

void build_nodal_wind_stencils(int N, double x0, double x1, const double* wind, std::vector<double>& q2,
                               std::vector<double>& q1) {
  convection_stencils(N, x0, x1, 3, wind, q2);
  convection_stencils(N, x0, x1, 2, wind, q1);
}

void build_level_tables(int N, double x0, double x1, std::vector<double>& q2, std::vector<double>& q1) {
  const int n2 = 2 * N + 1, n1 = N + 1;
  const double h = (x1 - x0) / N;
  q2.assign((size_t)4 * n2 * 5, 0.0);
  q1.assign((size_t)4 * n1 * 3, 0.0);
  double xi[3], w[3];
  gauss3(xi, w);
  for (int e = 0; e < N; ++e) {
    for (int q = 0; q < 3; ++q) {
      const double s = x0 + (e + xi[q]) * h;
      double v[3], d[3], lv[2], ld[2];
      quad_basis(xi[q], v, d);
      lin_basis(xi[q], lv, ld);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          const int row = 2 * e + a, off = (b - a) + 2;
          q2[((size_t)0 * n2 + row) * 5 + off] += w[q] * h * v[a] * v[b];
          q2[((size_t)1 * n2 + row) * 5 + off] += w[q] * d[a] * d[b] / h;
          q2[((size_t)2 * n2 + row) * 5 + off] += w[q] * v[a] * (1.0 - s * s) * d[b];
          q2[((size_t)3 * n2 + row) * 5 + off] += w[q] * h * v[a] * s * v[b];
        }
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          const int row = e + a, off = (b - a) + 1;
          q1[((size_t)0 * n1 + row) * 3 + off] += w[q] * h * lv[a] * lv[b];
          q1[((size_t)1 * n1 + row) * 3 + off] += w[q] * ld[a] * ld[b] / h;
          q1[((size_t)2 * n1 + row) * 3 + off] += w[q] * lv[a] * (1.0 - s * s) * ld[b];
          q1[((size_t)3 * n1 + row) * 3 + off] += w[q] * h * lv[a] * s * lv[b];
        }
    }
  }
}

void build_b_tables(int N, double x0, double x1, std::vector<double>& bt) {
  const int n2 = 2 * N + 1, n1 = N + 1;
  const double h = (x1 - x0) / N;
  // G1[n1][5], H1[n1][5], GT[n2][3], HT[n2][3]
  bt.assign((size_t)n1 * 10 + (size_t)n2 * 6, 0.0);
  double* G = bt.data();
  double* H = G + (size_t)n1 * 5;
  double* GT = H + (size_t)n1 * 5;
  double* HT = GT + (size_t)n2 * 3;
  double xi[3], w[3];
  gauss3(xi, w);
  for (int e = 0; e < N; ++e)
    for (int q = 0; q < 3; ++q) {
      double v[3], d[3], lv[2], ld[2];
      quad_basis(xi[q], v, d);
      lin_basis(xi[q], lv, ld);
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 3; ++b) {
          const int k = e + a, off = (b - 2 * a) + 2;  // Q2 node 2e+b relative to 2k
          G[(size_t)k * 5 + off] += w[q] * lv[a] * d[b];
          H[(size_t)k * 5 + off] += w[q] * h * lv[a] * v[b];
        }
    }
  for (int i = 0; i < n2; ++i)
    for (int t = 0; t < 3; ++t) {
      const int k = (i >> 1) - 1 + t;
      if (k < 0 || k >= n1) continue;
      const int off = i - 2 * k + 2;
      if (off < 0 || off > 4) continue;
      GT[(size_t)i * 3 + t] = G[(size_t)k * 5 + off];
      HT[(size_t)i * 3 + t] = H[(size_t)k * 5 + off];
    }
}

}  // namespace pint
