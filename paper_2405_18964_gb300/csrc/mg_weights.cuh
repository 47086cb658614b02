// mg_weights.cuh -- constant-coefficient stencil weights of the multigrid
// levels (internal).
#pragma once
#include "common.cuh"

namespace pint {

// ----------------------------------------------------------------------------
// Stencil weights.  On the uniform grid the 2-D weights of a constant-
// coefficient operator a M + b K depend only on the node type: for Q2 the
// parities of (ix, iy) (vertex / midpoint), for Q1 whether ix, iy lie on the
// boundary (natural conditions give half rows there).  They are formed in
// FP64 from the 1-D bands and rounded once to T; the convection part (which
// varies per node) comes from a per-node table built the same way.
// ----------------------------------------------------------------------------
template <int SP>
__device__ __forceinline__ int ntypes() { return SP == 2 ? 4 : 9; }
template <int SP>
__device__ __forceinline__ int nstencil() { return SP == 2 ? 25 : 9; }

// representative node index along one axis for a node type coordinate
template <int SP>
__device__ __forceinline__ int type_rep(int t, int n) {
  if (SP == 2) return t ? 1 : 2;           // midpoint : vertex
  return t == 0 ? 0 : (t == 1 ? 1 : n - 1);  // left boundary : interior : right boundary
}
template <int SP>
__device__ __forceinline__ int node_type(int ix, int iy, int n) {
  if (SP == 2) return (ix & 1) + 2 * (iy & 1);
  const int tx = ix == 0 ? 0 : (ix == n - 1 ? 2 : 1);
  const int ty = iy == 0 ? 0 : (iy == n - 1 ? 2 : 1);
  return tx + 3 * ty;
}

// Entry q = type * (stencil size) + k of level_weights: sw[q] = (a M + b K)
// at level l (FP64 -> T); sdi[type] = 1 / diagonal with the centre entry.
template <class T, int SP>
__device__ __forceinline__ void level_weight(const Tabs<double>& t64, int l, int n, cpx<double> a, double b, int q,
                                             cpx<T>* sw, cpx<T>* sdi) {
  constexpr int W = SP == 2 ? 5 : 3;
  const double* tab = SP == 2 ? t64.q2[l] : t64.q1[l];
  const int ns = nstencil<SP>();
  const int type = q / ns, k = q % ns;
  const int dx = k % W, dy = k / W;
  const int tx = SP == 2 ? (type & 1) : type % 3;
  const int ty = SP == 2 ? (type >> 1) : type / 3;
  const int ix = type_rep<SP>(tx, n), iy = type_rep<SP>(ty, n);
  const double mx = tab[(size_t)(0 * n + ix) * W + dx], my = tab[(size_t)(0 * n + iy) * W + dy];
  const double kx = tab[(size_t)(1 * n + ix) * W + dx], ky = tab[(size_t)(1 * n + iy) * W + dy];
  const double m2 = mx * my, k2 = kx * my + mx * ky;
  const cpx<double> w = mkc<double>(a.x * m2 + b * k2, a.y * m2);
  sw[q] = mkc<T>(T(w.x), T(w.y));
  if (k == ns / 2) {
    const double den = w.x * w.x + w.y * w.y;
    sdi[type] = mkc<T>(T(w.x / den), T(-w.y / den));
  }
}

// sw[type][k] = a M + b K at level l (FP64 -> T), sdi[type] = 1 / diagonal.
template <class T, int SP>
__device__ void level_weights(const Tabs<double>& t64, int l, int n, cpx<double> a, double b, cpx<T>* sw,
                              cpx<T>* sdi) {
  const int nt = ntypes<SP>(), ns = nstencil<SP>();
  for (int q = threadIdx.x; q < nt * ns; q += blockDim.x) level_weight<T, SP>(t64, l, n, a, b, q, sw, sdi);
}

// Row sum of a M on Q1 level l for one node type (FP64 -> T): the mass part
// only, the stiffness rows summing to zero.
template <class T>
__device__ __forceinline__ T level_rowsum_q1(const Tabs<double>& t64, int l, int n, double a, int type) {
  const double* tab = t64.q1[l];
  const int ix = type_rep<1>(type % 3, n), iy = type_rep<1>(type / 3, n);
  double sx = 0.0, sy = 0.0;
  for (int d = 0; d < 3; ++d) {
    sx += tab[(size_t)ix * 3 + d];
    sy += tab[(size_t)iy * 3 + d];
  }
  return T(a * sx * sy);
}
template <class T>
__device__ void level_rowsums_q1(const Tabs<double>& t64, int l, int n, double a, T* srs) {
  for (int type = threadIdx.x; type < 9; type += blockDim.x) srs[type] = level_rowsum_q1<T>(t64, l, n, a, type);
}

}  // namespace pint
