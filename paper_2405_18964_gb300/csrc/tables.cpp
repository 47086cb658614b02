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

}  // namespace

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
