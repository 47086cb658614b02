// common.cuh -- shared device types and matrix-free Q2/Q1 stencils.
//
// Every spatial operator of the paper (Sec. 2.2: M, L = nu K + N(w), B;
// Sec. 2.3: M_p, K_p, L_p) is, on the uniform tensor-product grid, a sum of
// Kronecker products of 1-D banded element matrices:
//   M   = M1 (x) M1
//   K   = K1 (x) M1 + M1 (x) K1
//   N   = 2 W1 (x) X1 - 2 X1 (x) W1      for w = (2y(1-x^2), -2x(1-y^2)),
//         W1_ik = int phi_i (1-s^2) phi_k',  X1_ik = int phi_i s phi_k
//   B   = -(G1 (x) H1, H1 (x) G1)        G1_ki = int psi_k phi_i', H1_ki = int psi_k phi_i
// (first factor acts on the x index, second on the y index).  The 1-D rows
// are stored per node as a band of 5 (Q2) or 3 (Q1) coefficients, so a
// 2-D stencil needs only the two 1-D rows of the node it updates.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define PINT_MAXLEV 12

template <class T>
struct alignas(2 * sizeof(T)) cpx {
  T x, y;
};

template <class T>
__host__ __device__ __forceinline__ cpx<T> mkc(T a, T b) {
  cpx<T> r;
  r.x = a;
  r.y = b;
  return r;
}
template <class T>
__host__ __device__ __forceinline__ cpx<T> czero() { return mkc<T>(T(0), T(0)); }
template <class T>
__host__ __device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return mkc<T>(a.x + b.x, a.y + b.y); }
template <class T>
__host__ __device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return mkc<T>(a.x - b.x, a.y - b.y); }
template <class T>
__host__ __device__ __forceinline__ cpx<T> operator*(cpx<T> a, cpx<T> b) {
  return mkc<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <class T>
__host__ __device__ __forceinline__ cpx<T> operator*(T s, cpx<T> a) { return mkc<T>(s * a.x, s * a.y); }
template <class T>
__host__ __device__ __forceinline__ cpx<T> conjc(cpx<T> a) { return mkc<T>(a.x, -a.y); }
// acc += s * v (real s)
template <class T>
__device__ __forceinline__ void rfma(cpx<T>& acc, T s, cpx<T> v) {
  acc.x = fma(s, v.x, acc.x);
  acc.y = fma(s, v.y, acc.y);
}
template <class T>
__device__ __forceinline__ cpx<T> cdiv(cpx<T> a, cpx<T> b) {
  T den = b.x * b.x + b.y * b.y;
  return mkc<T>((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}
template <class T, class U>
__host__ __device__ __forceinline__ cpx<T> ccast(cpx<U> a) { return mkc<T>(T(a.x), T(a.y)); }

__host__ __device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Per-level 1-D band tables of one precision.
//   q2[l]: [4][n2][5]  rows of M1, K1, W1, X1 on the Q2 node line of level l
//   q1[l]: [4][n1][3]  same on the Q1 node line
//   bt:    finest level only: G1[n1][5], H1[n1][5], GT[n2][3], HT[n2][3]
//          (GT/HT: the transposed bands, GT[i][t] = G1[k][i - 2k + 2] with
//           k = (i >> 1) - 1 + t, zero where k or the offset is invalid)
template <class T>
struct Tabs {
  int nlev;
  int N[PINT_MAXLEV];
  const T* q2[PINT_MAXLEV];
  const T* q1[PINT_MAXLEV];
  const T* bt;
};

// Operator coefficient set: A = a M + b K + c N (complex a; real b, c).
struct OpCoef {
  double ar, ai, b, c;
};

// ---------------------------------------------------------------------------
// Q2 scalar operator at node (ix, iy) of a grid with n2 nodes per side.
// Indices off the grid are clamped; their band coefficients are exactly 0.
// ---------------------------------------------------------------------------
template <class T, bool CONV>
__device__ __forceinline__ cpx<T> q2_op(const T* __restrict__ tab, int n2, int ix, int iy,
                                        const cpx<T>* __restrict__ x, cpx<T> a, T b, T c) {
  const T* Mx = tab + (size_t)(0 * n2 + ix) * 5;
  const T* Kx = tab + (size_t)(1 * n2 + ix) * 5;
  const T* My = tab + (size_t)(0 * n2 + iy) * 5;
  const T* Ky = tab + (size_t)(1 * n2 + iy) * 5;
  const T* Wx = tab + (size_t)(2 * n2 + ix) * 5;
  const T* Xx = tab + (size_t)(3 * n2 + ix) * 5;
  const T* Wy = tab + (size_t)(2 * n2 + iy) * 5;
  const T* Xy = tab + (size_t)(3 * n2 + iy) * 5;
  cpx<T> accM = czero<T>(), accK = czero<T>(), accN = czero<T>();
#pragma unroll
  for (int dy = 0; dy < 5; ++dy) {
    const int jy = clampi(iy + dy - 2, 0, n2 - 1);
    const cpx<T>* row = x + (size_t)jy * n2;
    cpx<T> sM = czero<T>(), sK = czero<T>(), sW = czero<T>(), sX = czero<T>();
#pragma unroll
    for (int dx = 0; dx < 5; ++dx) {
      const int jx = clampi(ix + dx - 2, 0, n2 - 1);
      const cpx<T> v = row[jx];
      rfma(sM, Mx[dx], v);
      rfma(sK, Kx[dx], v);
      if (CONV) {
        rfma(sW, Wx[dx], v);
        rfma(sX, Xx[dx], v);
      }
    }
    rfma(accM, My[dy], sM);
    rfma(accK, My[dy], sK);
    rfma(accK, Ky[dy], sM);
    if (CONV) {
      rfma(accN, Xy[dy], sW);
      rfma(accN, -Wy[dy], sX);
    }
  }
  cpx<T> r = a * accM;
  rfma(r, b, accK);
  if (CONV) rfma(r, T(2) * c, accN);
  return r;
}

// Q1 scalar operator at node (ix, iy) of a grid with n1 nodes per side:
// a (M1 x M1) + b (K1 x M1 + M1 x K1) + 2c (W1 x X1 - X1 x W1), evaluated
// separably.  The stiffness part uses that every row of the 1-D stiffness
// band sums to zero (Neumann rows included): sum_k K1_ik x_k =
// sum_k K1_ik (x_k - x_i).  The differences of neighbouring values are exact
// for smooth fields, so the near-null (nearly constant) component that the
// corner-pinned pressure Laplacian barely damps causes no cancellation.
template <class T, bool CONV>
__device__ __forceinline__ cpx<T> q1_op(const T* __restrict__ tab, int n1, int ix, int iy,
                                        const cpx<T>* __restrict__ x, cpx<T> a, T b, T c) {
  const T* Mx = tab + (size_t)(0 * n1 + ix) * 3;
  const T* Kx = tab + (size_t)(1 * n1 + ix) * 3;
  const T* My = tab + (size_t)(0 * n1 + iy) * 3;
  const T* Ky = tab + (size_t)(1 * n1 + iy) * 3;
  const T* Wx = tab + (size_t)(2 * n1 + ix) * 3;
  const T* Xx = tab + (size_t)(3 * n1 + ix) * 3;
  const T* Wy = tab + (size_t)(2 * n1 + iy) * 3;
  const T* Xy = tab + (size_t)(3 * n1 + iy) * 3;
  cpx<T> v[3][3];
#pragma unroll
  for (int dy = 0; dy < 3; ++dy) {
    const cpx<T>* row = x + (size_t)clampi(iy + dy - 1, 0, n1 - 1) * n1;
#pragma unroll
    for (int dx = 0; dx < 3; ++dx) v[dy][dx] = row[clampi(ix + dx - 1, 0, n1 - 1)];
  }
  cpx<T> accM = czero<T>(), accK = czero<T>(), accN = czero<T>();
#pragma unroll
  for (int dy = 0; dy < 3; ++dy) {
    cpx<T> sM = czero<T>(), sK = czero<T>(), sW = czero<T>(), sX = czero<T>();
#pragma unroll
    for (int dx = 0; dx < 3; ++dx) {
      rfma(sM, Mx[dx], v[dy][dx]);
      rfma(sK, Kx[dx], v[dy][dx] - v[dy][1]);
      if (CONV) {
        rfma(sW, Wx[dx], v[dy][dx]);
        rfma(sX, Xx[dx], v[dy][dx]);
      }
    }
    rfma(accM, My[dy], sM);
    rfma(accK, My[dy], sK);
    if (CONV) {
      rfma(accN, Xy[dy], sW);
      rfma(accN, -Wy[dy], sX);
    }
  }
#pragma unroll
  for (int dx = 0; dx < 3; ++dx) {
    cpx<T> tK = czero<T>();
#pragma unroll
    for (int dy = 0; dy < 3; ++dy) rfma(tK, Ky[dy], v[dy][dx] - v[1][dx]);
    rfma(accK, Mx[dx], tK);
  }
  cpx<T> r = a * accM;
  rfma(r, b, accK);
  if (CONV) rfma(r, T(2) * c, accN);
  return r;
}

// (B v)_k at Q1 node (kx, ky): -sum [G1 (x) H1] vx + [H1 (x) G1] vy.
template <class T>
__device__ __forceinline__ cpx<T> b_op(const T* __restrict__ bt, int n1, int n2, int kx, int ky,
                                       const cpx<T>* __restrict__ vx, const cpx<T>* __restrict__ vy) {
  const T* G = bt;
  const T* H = bt + (size_t)n1 * 5;
  const T* Gx = G + (size_t)kx * 5;
  const T* Hx = H + (size_t)kx * 5;
  const T* Gy = G + (size_t)ky * 5;
  const T* Hy = H + (size_t)ky * 5;
  cpx<T> acc = czero<T>();
#pragma unroll
  for (int dy = 0; dy < 5; ++dy) {
    const int jy = clampi(2 * ky + dy - 2, 0, n2 - 1);
    cpx<T> sx = czero<T>(), sy = czero<T>();
#pragma unroll
    for (int dx = 0; dx < 5; ++dx) {
      const int jx = clampi(2 * kx + dx - 2, 0, n2 - 1);
      rfma(sx, Gx[dx], vx[(size_t)jy * n2 + jx]);
      rfma(sy, Hx[dx], vy[(size_t)jy * n2 + jx]);
    }
    rfma(acc, Hy[dy], sx);
    rfma(acc, Gy[dy], sy);
  }
  return mkc<T>(-acc.x, -acc.y);
}

// (B^T p) at Q2 node (ix, iy): returns the x and y components.
template <class T>
__device__ __forceinline__ void bt_op(const T* __restrict__ bt, int n1, int n2, int ix, int iy,
                                      const cpx<T>* __restrict__ p, cpx<T>& ox, cpx<T>& oy) {
  const T* GT = bt + (size_t)n1 * 10;
  const T* HT = GT + (size_t)n2 * 3;
  const T* Gx = GT + (size_t)ix * 3;
  const T* Hx = HT + (size_t)ix * 3;
  const T* Gy = GT + (size_t)iy * 3;
  const T* Hy = HT + (size_t)iy * 3;
  cpx<T> ax = czero<T>(), ay = czero<T>();
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    const int ky = clampi((iy >> 1) - 1 + u, 0, n1 - 1);
    cpx<T> sg = czero<T>(), sh = czero<T>();
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const int kx = clampi((ix >> 1) - 1 + t, 0, n1 - 1);
      const cpx<T> v = p[(size_t)ky * n1 + kx];
      rfma(sg, Gx[t], v);
      rfma(sh, Hx[t], v);
    }
    rfma(ax, Hy[u], sg);
    rfma(ay, Gy[u], sh);
  }
  ox = mkc<T>(-ax.x, -ax.y);
  oy = mkc<T>(-ay.x, -ay.y);
}

// Real-valued variants for the FP64 time-domain KKT matvec reuse the complex
// ones through a zero imaginary part; they are not on the hot path.

// Index of Q2 node (ix, iy) in the class-blocked layout of a grid with n2
// nodes per side: 36 residue classes (ix mod 6, iy mod 6) of w6 x w6 nodes,
// w6 = ceil(n2 / 6).  The per-node convection tables use this order.
__host__ __device__ __forceinline__ long long q2_blocked_index(int n2, int ix, int iy) {
  const long long w6 = (n2 + 5) / 6;
  return ((ix % 6) + 6 * (iy % 6)) * w6 * w6 + (iy / 6) * w6 + ix / 6;
}

// Convection from a per-node stencil row (W x W, rounded once from FP64):
// sum_k row[k] x[neighbour k], neighbours clamped (their row entries are 0).
template <class T, int W>
__device__ __forceinline__ cpx<T> conv_row(const T* __restrict__ row, int n, int ix, int iy,
                                           const cpx<T>* __restrict__ x) {
  constexpr int H = W / 2;
  cpx<T> acc = czero<T>();
#pragma unroll
  for (int dy = 0; dy < W; ++dy) {
    const cpx<T>* r = x + (size_t)clampi(iy + dy - H, 0, n - 1) * n;
#pragma unroll
    for (int dx = 0; dx < W; ++dx) rfma(acc, row[dy * W + dx], r[clampi(ix + dx - H, 0, n - 1)]);
  }
  return acc;
}

__device__ __forceinline__ bool q2_interior(int ix, int iy, int n2) {
  return ix > 0 && iy > 0 && ix < n2 - 1 && iy < n2 - 1;
}
__device__ __forceinline__ bool q1_free(int ix, int iy) { return (ix | iy) != 0; }
