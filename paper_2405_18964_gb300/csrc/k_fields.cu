// k_fields.cu -- field-wise kernels: the FP64 KKT matvec (Eq. FinalA), the
// frequency-block matvec (Eq. SubBlockG / Z_j of Eq. GJTransformation),
// operator combinations used by Uzawa (Eq. Uzawa11) and Algorithm 3, the
// Stokes transforms (T_j^l)^{-1}, (T_j^r)^{-1}, and the time DFT (Sec. 3.1).
#include "fields.h"

namespace pint {

namespace {

constexpr int TPB = 256;

// Real-valued 5x5 sums of one Q2 field: M x, K x, and the two convection
// partial sums (N x = 2 * nn).
template <bool CONV>
__device__ __forceinline__ void q2_mkn_r(const double* __restrict__ tab, int n2, int ix, int iy,
                                         const double* __restrict__ x, double& m, double& k, double& nn) {
  const double* Mx = tab + (size_t)(0 * n2 + ix) * 5;
  const double* Kx = tab + (size_t)(1 * n2 + ix) * 5;
  const double* Wx = tab + (size_t)(2 * n2 + ix) * 5;
  const double* Xx = tab + (size_t)(3 * n2 + ix) * 5;
  const double* My = tab + (size_t)(0 * n2 + iy) * 5;
  const double* Ky = tab + (size_t)(1 * n2 + iy) * 5;
  const double* Wy = tab + (size_t)(2 * n2 + iy) * 5;
  const double* Xy = tab + (size_t)(3 * n2 + iy) * 5;
  m = k = nn = 0.0;
#pragma unroll
  for (int dy = 0; dy < 5; ++dy) {
    const double* row = x + (size_t)clampi(iy + dy - 2, 0, n2 - 1) * n2;
    double sM = 0, sK = 0, sW = 0, sX = 0;
#pragma unroll
    for (int dx = 0; dx < 5; ++dx) {
      const double v = row[clampi(ix + dx - 2, 0, n2 - 1)];
      sM = fma(Mx[dx], v, sM);
      sK = fma(Kx[dx], v, sK);
      if (CONV) {
        sW = fma(Wx[dx], v, sW);
        sX = fma(Xx[dx], v, sX);
      }
    }
    m = fma(My[dy], sM, m);
    k = fma(My[dy], sK, k);
    k = fma(Ky[dy], sM, k);
    if (CONV) {
      nn = fma(Xy[dy], sW, nn);
      nn = fma(-Wy[dy], sX, nn);
    }
  }
  nn *= 2.0;
}

// One row of a node-order convection stencil applied to a Q2 field at an
// interior node.  Offsets that leave the grid (+-2 from a midside node next to
// the boundary) are clamped; their stencil entries are zero.
__device__ __forceinline__ double conv_row_r(const double* __restrict__ st, int n2, int ix, int iy,
                                             const double* __restrict__ x) {
  double acc = 0.0;
#pragma unroll
  for (int dy = 0; dy < 5; ++dy) {
    const double* row = x + (size_t)clampi(iy + dy - 2, 0, n2 - 1) * n2;
#pragma unroll
    for (int dx = 0; dx < 5; ++dx) acc = fma(st[dy * 5 + dx], row[clampi(ix + dx - 2, 0, n2 - 1)], acc);
  }
  return acc;
}

__device__ __forceinline__ void bt_op_r(const double* __restrict__ bt, int n1, int n2, int ix, int iy,
                                        const double* __restrict__ p, double& ox, double& oy) {
  const double* GT = bt + (size_t)n1 * 10;
  const double* HT = GT + (size_t)n2 * 3;
  double ax = 0, ay = 0;
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    const int ky = clampi((iy >> 1) - 1 + u, 0, n1 - 1);
    double sg = 0, sh = 0;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const double v = p[(size_t)ky * n1 + clampi((ix >> 1) - 1 + t, 0, n1 - 1)];
      sg = fma(GT[ix * 3 + t], v, sg);
      sh = fma(HT[ix * 3 + t], v, sh);
    }
    ax = fma(HT[iy * 3 + u], sg, ax);
    ay = fma(GT[iy * 3 + u], sh, ay);
  }
  ox = -ax;
  oy = -ay;
}

__device__ __forceinline__ double b_op_r(const double* __restrict__ bt, int n1, int n2, int kx, int ky,
                                         const double* __restrict__ vx, const double* __restrict__ vy) {
  const double* G = bt;
  const double* H = bt + (size_t)n1 * 5;
  double acc = 0;
#pragma unroll
  for (int dy = 0; dy < 5; ++dy) {
    const int jy = clampi(2 * ky + dy - 2, 0, n2 - 1);
    double sx = 0, sy = 0;
#pragma unroll
    for (int dx = 0; dx < 5; ++dx) {
      const int jx = clampi(2 * kx + dx - 2, 0, n2 - 1);
      sx = fma(G[kx * 5 + dx], vx[(size_t)jy * n2 + jx], sx);
      sy = fma(H[kx * 5 + dx], vy[(size_t)jy * n2 + jx], sy);
    }
    acc = fma(H[ky * 5 + dy], sx, acc);
    acc = fma(G[ky * 5 + dy], sy, acc);
  }
  return -acc;
}

template <bool CONV>
__global__ void __launch_bounds__(TPB) kkt_q2_kernel(KKTArgs A) {
  const int ns = A.s.ns, n2 = A.s.n2, n1 = A.s.n1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (t >= ns) return;
  const int ix = t % n2, iy = t / n2;
  const long long nb = A.s.nblk;
  const double* X = A.x + (size_t)k * nb;
  double* Y = A.y + (size_t)k * nb;
  if (!q2_interior(ix, iy, n2)) {
    Y[A.s.vx + t] = 0.0;
    Y[A.s.vy + t] = 0.0;
    Y[A.s.lx + t] = 0.0;
    Y[A.s.ly + t] = 0.0;
    return;
  }
  const bool has_next = k + 1 < A.K, has_prev = k > 0;
  const double* Xn = has_next ? X + nb : X;
  const double* Xp = has_prev ? X - nb : X;
  const double fn = has_next ? 1.0 : 0.0, fp = has_prev ? 1.0 : 0.0;
  const double tau = A.tau, tb = A.tau / A.beta, nu = A.nu;
  const double* tab = A.tabs.q2[0];
  const double* Mx = tab + (size_t)(0 * n2 + ix) * 5;
  const double* My = tab + (size_t)(0 * n2 + iy) * 5;
  double btm_x, btm_y, btp_x, btp_y;
  bt_op_r(A.tabs.bt, n1, n2, ix, iy, X + A.s.mu, btm_x, btm_y);
  bt_op_r(A.tabs.bt, n1, n2, ix, iy, X + A.s.p, btp_x, btp_y);
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const long long sv = c ? A.s.vy : A.s.vx, sl = c ? A.s.ly : A.s.lx;
    const double* v = X + sv;
    const double* l = X + sl;
    const double* l1 = Xn + sl;
    const double* vm = Xp + sv;
    // M applied to the two time-coupled combinations
    double m1 = 0, m2 = 0;
#pragma unroll
    for (int dy = 0; dy < 5; ++dy) {
      const size_t r = (size_t)clampi(iy + dy - 2, 0, n2 - 1) * n2;
      double s1 = 0, s2 = 0;
#pragma unroll
      for (int dx = 0; dx < 5; ++dx) {
        const size_t q = r + clampi(ix + dx - 2, 0, n2 - 1);
        const double lv = l[q];
        const double a1 = tau * v[q] + lv - fn * l1[q];
        const double a2 = v[q] - fp * vm[q] - tb * lv;
        s1 = fma(Mx[dx], a1, s1);
        s2 = fma(Mx[dx], a2, s2);
      }
      m1 = fma(My[dy], s1, m1);
      m2 = fma(My[dy], s2, m2);
    }
    double mv, kv, nv, ml, kl, nl;
    q2_mkn_r<CONV>(tab, n2, ix, iy, v, mv, kv, nv);
    q2_mkn_r<CONV>(tab, n2, ix, iy, l, ml, kl, nl);
    if (A.nst) {
      nv = conv_row_r(A.nst + (size_t)t * 25, n2, ix, iy, v);
      nl = conv_row_r(A.nst + (size_t)t * 25, n2, ix, iy, l);
    }
    // adjoint rows: tau M v_k + M lam_k - M lam_{k+1} + tau L^T lam_k + tau B^T mu_k
    Y[sv + t] = m1 + tau * (nu * kl - nl) + tau * (c ? btm_y : btm_x);
    // state rows: M v_k - M v_{k-1} + tau L v_k + tau B^T p_k - tau/beta M lam_k
    Y[sl + t] = m2 + tau * (nu * kv + nv) + tau * (c ? btp_y : btp_x);
  }
}

__global__ void __launch_bounds__(TPB) kkt_q1_kernel(KKTArgs A) {
  const int nq = A.s.nq, n1 = A.s.n1, n2 = A.s.n2;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (t >= nq) return;
  const int kx = t % n1, ky = t / n1;
  const long long nb = A.s.nblk;
  const double* X = A.x + (size_t)k * nb;
  double* Y = A.y + (size_t)k * nb;
  if (!q1_free(kx, ky)) {
    Y[A.s.p + t] = 0.0;
    Y[A.s.mu + t] = 0.0;
    return;
  }
  Y[A.s.p + t] = A.tau * b_op_r(A.tabs.bt, n1, n2, kx, ky, X + A.s.lx, X + A.s.ly);
  Y[A.s.mu + t] = A.tau * b_op_r(A.tabs.bt, n1, n2, kx, ky, X + A.s.vx, X + A.s.vy);
}

// ---------------------------------------------------------------------------
// complex M, K, N sums of one Q2 field
template <class T, bool CONV>
__device__ __forceinline__ void q2_mkn_c(const T* __restrict__ tab, int n2, int ix, int iy,
                                         const cpx<T>* __restrict__ x, cpx<T>& m, cpx<T>& k, cpx<T>& nn,
                                         const T* __restrict__ nrow) {
  const T* Mx = tab + (size_t)(0 * n2 + ix) * 5;
  const T* Kx = tab + (size_t)(1 * n2 + ix) * 5;
  const T* My = tab + (size_t)(0 * n2 + iy) * 5;
  const T* Ky = tab + (size_t)(1 * n2 + iy) * 5;
  m = k = nn = czero<T>();
#pragma unroll
  for (int dy = 0; dy < 5; ++dy) {
    const cpx<T>* row = x + (size_t)clampi(iy + dy - 2, 0, n2 - 1) * n2;
    cpx<T> sM = czero<T>(), sK = czero<T>();
#pragma unroll
    for (int dx = 0; dx < 5; ++dx) {
      const cpx<T> v = row[clampi(ix + dx - 2, 0, n2 - 1)];
      rfma(sM, Mx[dx], v);
      rfma(sK, Kx[dx], v);
      if (CONV) rfma(nn, nrow[dy * 5 + dx], v);
    }
    rfma(m, My[dy], sM);
    rfma(k, My[dy], sK);
    rfma(k, Ky[dy], sM);
  }
}

template <class T, bool CONV>
__global__ void __launch_bounds__(TPB) blk_q2_kernel(BlkArgs<T> A) {
  const int ns = A.s.ns, n2 = A.s.n2, n1 = A.s.n1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (t >= ns) return;
  if (A.active && !A.active[j]) return;
  const int ix = t % n2, iy = t / n2;
  const long long nb = A.s.nblk;
  const cpx<T>* X = A.x + (size_t)j * nb;
  cpx<T>* Y = A.y + (size_t)j * nb;
  if (!q2_interior(ix, iy, n2)) {
    Y[A.s.vx + t] = czero<T>();
    Y[A.s.vy + t] = czero<T>();
    Y[A.s.lx + t] = czero<T>();
    Y[A.s.ly + t] = czero<T>();
    return;
  }
  const BlkCoef cf = A.coef[j];
  const cpx<T> a11 = mkc<T>(T(cf.a11r), T(cf.a11i)), a12 = mkc<T>(T(cf.a12r), T(cf.a12i));
  const cpx<T> a21 = mkc<T>(T(cf.a21r), T(cf.a21i)), a22 = mkc<T>(T(cf.a22r), T(cf.a22i));
  const T g12 = T(cf.g12), g21 = T(cf.g21), dl = T(cf.dl), nu = T(A.nu);
  const T* tab = A.tabs.q2[0];
  cpx<T> bmx, bmy, bpx, bpy;
  const T* nrow = CONV ? A.n2d + (size_t)q2_blocked_index(n2, ix, iy) * 25 : nullptr;
  bt_op<T>(A.tabs.bt, n1, n2, ix, iy, X + A.s.mu, bmx, bmy);
  bt_op<T>(A.tabs.bt, n1, n2, ix, iy, X + A.s.p, bpx, bpy);
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const long long sv = c ? A.s.vy : A.s.vx, sl = c ? A.s.ly : A.s.lx;
    cpx<T> mv, kv, nv, ml, kl, nl;
    q2_mkn_c<T, CONV>(tab, n2, ix, iy, X + sv, mv, kv, nv, nrow);
    q2_mkn_c<T, CONV>(tab, n2, ix, iy, X + sl, ml, kl, nl, nrow);
    cpx<T> r1 = a11 * mv + a12 * ml;
    cpx<T> lt = nu * kl;
    if (CONV) lt = lt - nl;
    rfma(r1, g12, lt);
    rfma(r1, dl, c ? bmy : bmx);
    cpx<T> r2 = a21 * mv + a22 * ml;
    cpx<T> lv = nu * kv;
    if (CONV) lv = lv + nv;
    rfma(r2, g21, lv);
    rfma(r2, dl, c ? bpy : bpx);
    Y[sv + t] = r1;
    Y[sl + t] = r2;
  }
}

template <class T>
__global__ void __launch_bounds__(TPB) blk_q1_kernel(BlkArgs<T> A) {
  const int nq = A.s.nq, n1 = A.s.n1, n2 = A.s.n2;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (t >= nq) return;
  if (A.active && !A.active[j]) return;
  const int kx = t % n1, ky = t / n1;
  const long long nb = A.s.nblk;
  const cpx<T>* X = A.x + (size_t)j * nb;
  cpx<T>* Y = A.y + (size_t)j * nb;
  if (!q1_free(kx, ky)) {
    Y[A.s.p + t] = czero<T>();
    Y[A.s.mu + t] = czero<T>();
    return;
  }
  const T dl = T(A.coef[j].dl);
  Y[A.s.p + t] = dl * b_op<T>(A.tabs.bt, n1, n2, kx, ky, X + A.s.lx, X + A.s.ly);
  Y[A.s.mu + t] = dl * b_op<T>(A.tabs.bt, n1, n2, kx, ky, X + A.s.vx, X + A.s.vy);
}

// ---------------------------------------------------------------------------
template <class T, int SP, bool CONV>
__global__ void __launch_bounds__(TPB) combo_kernel(ComboArgs<T> A) {
  const int n = SP == 2 ? A.s.n2 : A.s.n1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (t >= n * n) return;
  if (A.active && !A.active[j]) return;
  const int ix = t % n, iy = t / n;
  const long long nb = A.s.nblk;
  const cpx<T>* X = A.x + (size_t)j * nb;
  const cpx<T>* Z = A.z ? A.z + (size_t)j * nb : nullptr;
  cpx<T>* O = A.out + (size_t)j * nb;
  const bool unk = SP == 2 ? q2_interior(ix, iy, n) : q1_free(ix, iy);
  const OpCoef* cf = A.coef + (size_t)j * A.ncoef;
  const T* tab = SP == 2 ? A.tabs.q2[0] : A.tabs.q1[0];
  const T* nrow = nullptr;
  if (CONV) nrow = SP == 2 ? A.n2d + (size_t)q2_blocked_index(n, ix, iy) * 25 : A.np2d + (size_t)t * 9;
  for (int r = 0; r < A.nrows; ++r) {
    const ComboRow& R = A.rows[r];
    cpx<T> acc = czero<T>();
    if (unk) {
      if (R.has_z) acc = mkc<T>(T(cf[R.zc].ar), T(cf[R.zc].ai)) * Z[R.z_slot + t];
      for (int q = 0; q < R.nt; ++q) {
        const OpCoef oc = cf[R.tc[q]];
        const cpx<T> a = mkc<T>(T(oc.ar), T(oc.ai));
        const cpx<T>* xin = X + R.in_slot[q];
        if (SP == 2) {
          acc = acc + q2_op<T, false>(tab, n, ix, iy, xin, a, T(oc.b), T(0));
          if (CONV && oc.c != 0.0) rfma(acc, T(oc.c), conv_row<T, 5>(nrow, n, ix, iy, xin));
        } else {
          acc = acc + q1_op<T, false>(tab, n, ix, iy, xin, a, T(oc.b), T(0));
          if (CONV && oc.c != 0.0) rfma(acc, T(oc.c), conv_row<T, 3>(nrow, n, ix, iy, xin));
        }
      }
    }
    O[R.out_slot + t] = acc;
  }
}

template <class T>
__global__ void __launch_bounds__(TPB) bres_kernel(BResArgs<T> A) {
  const int nq = A.s.nq, n1 = A.s.n1, n2 = A.s.n2;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (t >= nq) return;
  if (A.active && !A.active[j]) return;
  const int kx = t % n1, ky = t / n1;
  const long long nb = A.s.nblk;
  const cpx<T>* X = A.x + (size_t)j * nb;
  const cpx<T>* Z = A.z + (size_t)j * nb;
  cpx<T>* O = A.out + (size_t)j * nb;
  if (!q1_free(kx, ky)) {
    O[A.out0 + t] = czero<T>();
    O[A.out1 + t] = czero<T>();
    return;
  }
  const T c = T(A.cj ? A.cj[j] : A.c);
  cpx<T> r0 = Z[A.z0 + t], r1 = Z[A.z1 + t];
  rfma(r0, c, b_op<T>(A.tabs.bt, n1, n2, kx, ky, X + A.vel0, X + A.vel0 + A.s.ns));
  rfma(r1, c, b_op<T>(A.tabs.bt, n1, n2, kx, ky, X + A.vel1, X + A.vel1 + A.s.ns));
  O[A.out0 + t] = r0;
  O[A.out1 + t] = r1;
}

template <class T>
__global__ void lincomb_kernel(int J, long long nblk, long long len, cpx<T>* out, long long so, const cpx<T>* A,
                               long long sa, const double* al, const cpx<T>* B, long long sb, const double* be,
                               const int* active) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= len) return;
  if (active && !active[j]) return;
  const cpx<T> a = mkc<T>(T(al[2 * j]), T(al[2 * j + 1]));
  cpx<T> r = a * A[(size_t)j * nblk + sa + i];
  if (B) r = r + mkc<T>(T(be[2 * j]), T(be[2 * j + 1])) * B[(size_t)j * nblk + sb + i];
  out[(size_t)j * nblk + so + i] = r;
}

// i * z
template <class T>
__device__ __forceinline__ cpx<T> mul_i(cpx<T> z) { return mkc<T>(-z.y, z.x); }

template <class T>
__global__ void stokes_transform_kernel(int dir, int J, Slots s, const double* tc, cpx<T>* X) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  const long long nv = 2LL * s.ns;
  if (i >= nv + s.nq) return;
  const T sq = T(tc[3 * j]), dc = T(tc[3 * j + 1]), c2 = T(tc[3 * j + 2]);
  cpx<T>* B = X + (size_t)j * s.nblk;
  if (i < nv) {  // velocity-type pair: block 1 (v slots) and block 2 (lambda slots)
    const long long p1 = (i < s.ns ? s.vx + i : s.vy + (i - s.ns));
    const long long p2 = (i < s.ns ? s.lx + i : s.ly + (i - s.ns));
    const cpx<T> r1 = B[p1], r2 = B[p2];
    if (dir == 0) {  // (T^l)^{-1}: s1 = r1/s, s2 = (r2 - i dc/s s1) c2/s
      const cpx<T> s1 = (T(1) / sq) * r1;
      const cpx<T> s2 = (c2 / sq) * (r2 - (dc / sq) * mul_i(s1));
      B[p1] = s1;
      B[p2] = s2;
    } else {  // (T^r)^{-1}: y2 = x2 c2/s, y1 = (x1 + i dc/s y2)/s
      const cpx<T> y2 = (c2 / sq) * r2;
      const cpx<T> y1 = (T(1) / sq) * (r1 + (dc / sq) * mul_i(y2));
      B[p1] = y1;
      B[p2] = y2;
    }
  } else {  // pressure-type pair: block 3 (p slot) and block 4 (mu slot)
    const long long q = i - nv;
    const cpx<T> r3 = B[s.p + q], r4 = B[s.mu + q];
    if (dir == 0) {  // s3 = r3/(s c2), s4 = (r4 - i dc c2/s s3)/s
      const cpx<T> s3 = (T(1) / (sq * c2)) * r3;
      const cpx<T> s4 = (T(1) / sq) * (r4 - (dc * c2 / sq) * mul_i(s3));
      B[s.p + q] = s3;
      B[s.mu + q] = s4;
    } else {  // y4 = x4/s, y3 = (x3 + i dc c2/s y4)/(s c2)
      const cpx<T> y4 = (T(1) / sq) * r4;
      const cpx<T> y3 = (T(1) / (sq * c2)) * (r3 + (dc * c2 / sq) * mul_i(y4));
      B[s.p + q] = y3;
      B[s.mu + q] = y4;
    }
  }
}

// ---------------------------------------------------------------------------
// Time DFT.  A CTA stages a tile of DFT_COLS spatial columns for all K time
// levels in shared memory; each thread then produces outputs for one column
// and a strided subset of frequencies (forward) / time levels (inverse).
constexpr int DFT_COLS = 32;
constexpr int DFT_THREADS = 256;

template <class T>
__global__ void __launch_bounds__(DFT_THREADS) dft_fwd_kernel(int K, int J, long long nblk, const double* __restrict__ x,
                                                              cpx<T>* __restrict__ X, const T* __restrict__ cosk,
                                                              const T* __restrict__ sink) {
  extern __shared__ unsigned char smem_raw[];
  T* xs = reinterpret_cast<T*>(smem_raw);  // [K][DFT_COLS]
  T* cs = xs + (size_t)K * DFT_COLS;       // [K]
  T* sn = cs + K;                          // [K]
  const long long col0 = (long long)blockIdx.x * DFT_COLS;
  for (int idx = threadIdx.x; idx < K * DFT_COLS; idx += blockDim.x) {
    const int k = idx / DFT_COLS, c = idx % DFT_COLS;
    const long long col = col0 + c;
    xs[idx] = col < nblk ? T(x[(size_t)k * nblk + col]) : T(0);
  }
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    cs[k] = cosk[k];
    sn[k] = sink[k];
  }
  __syncthreads();
  const int c = threadIdx.x % DFT_COLS;
  const int grp = threadIdx.x / DFT_COLS;
  constexpr int NG = DFT_THREADS / DFT_COLS;
  const long long col = col0 + c;
  for (int j = grp; j < J; j += NG) {
    T re = 0, im = 0;
    int m = 0;
    for (int k = 0; k < K; ++k) {
      const T v = xs[k * DFT_COLS + c];
      re = fma(v, cs[m], re);
      im = fma(-v, sn[m], im);
      m += j;
      if (m >= K) m -= K;
    }
    if (col < nblk) X[(size_t)j * nblk + col] = mkc<T>(re, im);
  }
}

template <class T>
__global__ void __launch_bounds__(DFT_THREADS) dft_inv_kernel(int K, int J, long long nblk,
                                                              const cpx<T>* __restrict__ X, double* __restrict__ y,
                                                              const T* __restrict__ cosk,
                                                              const T* __restrict__ sink) {
  extern __shared__ unsigned char smem_raw[];
  cpx<T>* xs = reinterpret_cast<cpx<T>*>(smem_raw);  // [J][DFT_COLS]
  T* cs = reinterpret_cast<T*>(xs + (size_t)J * DFT_COLS);
  T* sn = cs + K;
  const long long col0 = (long long)blockIdx.x * DFT_COLS;
  const T invK = T(1) / T(K);
  for (int idx = threadIdx.x; idx < J * DFT_COLS; idx += blockDim.x) {
    const int j = idx / DFT_COLS, c = idx % DFT_COLS;
    const long long col = col0 + c;
    // weight 1 for j = 0 and (K even) j = K/2, else 2 (conjugate pair)
    const T w = (j == 0 || 2 * j == K) ? invK : T(2) * invK;
    cpx<T> v = col < nblk ? X[(size_t)j * nblk + col] : czero<T>();
    xs[idx] = w * v;
  }
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    cs[k] = cosk[k];
    sn[k] = sink[k];
  }
  __syncthreads();
  const int c = threadIdx.x % DFT_COLS;
  const int grp = threadIdx.x / DFT_COLS;
  constexpr int NG = DFT_THREADS / DFT_COLS;
  const long long col = col0 + c;
  for (int k = grp; k < K; k += NG) {
    T acc = 0;
    int m = 0;
    for (int j = 0; j < J; ++j) {
      const cpx<T> v = xs[j * DFT_COLS + c];
      // Re(v e^{+2 pi i j k / K})
      acc = fma(v.x, cs[m], acc);
      acc = fma(-v.y, sn[m], acc);
      m += k;
      if (m >= K) m -= K;
    }
    if (col < nblk) y[(size_t)k * nblk + col] = (double)acc;
  }
}

__global__ void mask_kernel(Slots s, long long nvec, int ncomp, double* x) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per = s.nblk;
  if (i >= nvec * per) return;
  const long long o = i % per;
  bool keep;
  long long q;
  if (o < 2LL * s.ns) {
    q = o % s.ns;
    keep = q2_interior((int)(q % s.n2), (int)(q / s.n2), s.n2);
  } else if (o < 2LL * s.ns + s.nq) {
    keep = (o - 2LL * s.ns) != 0;
  } else if (o < 4LL * s.ns + s.nq) {
    q = (o - 2LL * s.ns - s.nq) % s.ns;
    keep = q2_interior((int)(q % s.n2), (int)(q / s.n2), s.n2);
  } else {
    keep = (o - 4LL * s.ns - s.nq) != 0;
  }
  if (!keep)
    for (int c = 0; c < ncomp; ++c) x[i * ncomp + c] = 0.0;
}

__global__ void d2f_kernel(const double* a, float* b, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}
__global__ void f2d_kernel(const float* a, double* b, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}
__global__ void nonfinite_kernel(const double* a, long long n, int* count) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !isfinite(a[i])) atomicAdd(count, 1);
}

// M applied to a Q2 field whose non-interior nodal values are treated as 0.
__device__ __forceinline__ double mass_interior(const double* tab, int n2, int ix, int iy, const double* x) {
  const double* Mx = tab + (size_t)ix * 5;
  const double* My = tab + (size_t)iy * 5;
  double acc = 0.0;
  for (int dy = 0; dy < 5; ++dy) {
    const int jy = iy + dy - 2;
    if (jy <= 0 || jy >= n2 - 1) continue;
    double s = 0.0;
    for (int dx = 0; dx < 5; ++dx) {
      const int jx = ix + dx - 2;
      if (jx <= 0 || jx >= n2 - 1) continue;
      s = fma(Mx[dx], x[(size_t)jy * n2 + jx], s);
    }
    acc = fma(My[dy], s, acc);
  }
  return acc;
}

// M applied to a Q2 field at an interior node, every nodal value included
// (the full mass row M_{I,:}).  Out-of-range stencil offsets only occur for
// midside nodes, whose +-2 band entries are zero.
__device__ __forceinline__ double mass_all(const double* tab, int n2, int ix, int iy, const double* x) {
  const double* Mx = tab + (size_t)ix * 5;
  const double* My = tab + (size_t)iy * 5;
  double acc = 0.0;
  for (int dy = 0; dy < 5; ++dy) {
    const size_t r = (size_t)clampi(iy + dy - 2, 0, n2 - 1) * n2;
    double s = 0.0;
    for (int dx = 0; dx < 5; ++dx) s = fma(Mx[dx], x[r + clampi(ix + dx - 2, 0, n2 - 1)], s);
    acc = fma(My[dy], s, acc);
  }
  return acc;
}

__device__ __forceinline__ double mass_load(bool full, const double* tab, int n2, int ix, int iy, const double* x) {
  return full ? mass_all(tab, n2, ix, iy, x) : mass_interior(tab, n2, ix, iy, x);
}

__global__ void lift_scatter_kernel(Slots s, int K, const double* __restrict__ g, double* __restrict__ x) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (i >= s.ns || k >= K) return;
  const int ix = (int)(i % s.n2), iy = (int)(i / s.n2);
  if (q2_interior(ix, iy, s.n2)) return;
  double* X = x + (size_t)k * s.nblk;
  X[s.vx + i] = g[((size_t)k * 2 + 0) * s.ns + i];
  X[s.vy + i] = g[((size_t)k * 2 + 1) * s.ns + i];
}

__global__ void rhs_kernel(RhsArgs A) {
  const int ns = A.s.ns, n2 = A.s.n2, nq = A.s.nq;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  double* B = A.b + (size_t)k * A.s.nblk;
  if (t < nq) {
    B[A.s.p + t] = 0.0;
    B[A.s.mu + t] = 0.0;
  }
  if (t >= ns) return;
  const int ix = (int)(t % n2), iy = (int)(t / n2);
  const bool inner = q2_interior(ix, iy, n2);
  const double* tab = A.tabs.q2[0];
  for (int c = 0; c < 2; ++c) {
    double bv = 0.0, bl = 0.0;
    if (inner) {
      const bool fl = A.full != 0;
      bv = A.tau * mass_load(fl, tab, n2, ix, iy, A.vd + ((size_t)k * 2 + c) * ns);
      if (A.f) bl = A.tau * mass_load(fl, tab, n2, ix, iy, A.f + ((size_t)k * 2 + c) * ns);
      if (A.v0 && k == 0) bl += mass_load(fl, tab, n2, ix, iy, A.v0 + (size_t)c * ns);
    }
    B[(c ? A.s.vy : A.s.vx) + t] = bv;
    B[(c ? A.s.ly : A.s.lx) + t] = bl;
  }
}

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

void launch_rhs(const RhsArgs& a, cudaStream_t st) {
  const long long n = a.s.ns > a.s.nq ? a.s.ns : a.s.nq;
  rhs_kernel<<<dim3(blocks_for(n, TPB), a.K), TPB, 0, st>>>(a);
}

void launch_lift_scatter(const Slots& s, int K, const double* g, double* x, cudaStream_t st) {
  lift_scatter_kernel<<<dim3(blocks_for(s.ns, TPB), K), TPB, 0, st>>>(s, K, g, x);
}

// ============================ launchers ====================================
void launch_kkt_matvec(const KKTArgs& a, cudaStream_t st) {
  dim3 g2(blocks_for(a.s.ns, TPB), a.K), g1(blocks_for(a.s.nq, TPB), a.K);
  if (a.conv)
    kkt_q2_kernel<true><<<g2, TPB, 0, st>>>(a);
  else
    kkt_q2_kernel<false><<<g2, TPB, 0, st>>>(a);
  kkt_q1_kernel<<<g1, TPB, 0, st>>>(a);
}

template <class T>
void launch_block_matvec(const BlkArgs<T>& a, cudaStream_t st) {
  dim3 g2(blocks_for(a.s.ns, TPB), a.J), g1(blocks_for(a.s.nq, TPB), a.J);
  if (a.conv)
    blk_q2_kernel<T, true><<<g2, TPB, 0, st>>>(a);
  else
    blk_q2_kernel<T, false><<<g2, TPB, 0, st>>>(a);
  blk_q1_kernel<T><<<g1, TPB, 0, st>>>(a);
}

template <class T>
void launch_combo(const ComboArgs<T>& a, cudaStream_t st) {
  const int n = a.space == 2 ? a.s.n2 : a.s.n1;
  dim3 g(blocks_for((long long)n * n, TPB), a.J);
  if (a.space == 2) {
    if (a.conv)
      combo_kernel<T, 2, true><<<g, TPB, 0, st>>>(a);
    else
      combo_kernel<T, 2, false><<<g, TPB, 0, st>>>(a);
  } else {
    if (a.conv)
      combo_kernel<T, 1, true><<<g, TPB, 0, st>>>(a);
    else
      combo_kernel<T, 1, false><<<g, TPB, 0, st>>>(a);
  }
}

template <class T>
void launch_bres(const BResArgs<T>& a, cudaStream_t st) {
  dim3 g(blocks_for(a.s.nq, TPB), a.J);
  bres_kernel<T><<<g, TPB, 0, st>>>(a);
}

template <class T>
void launch_lincomb(int J, long long nblk, long long len, cpx<T>* out, long long so, const cpx<T>* A, long long sa,
                    const double* al, const cpx<T>* B, long long sb, const double* be, const int* active,
                    cudaStream_t st) {
  dim3 g(blocks_for(len, TPB), J);
  lincomb_kernel<T><<<g, TPB, 0, st>>>(J, nblk, len, out, so, A, sa, al, B, sb, be, active);
}

template <class T>
void launch_stokes_transform(int dir, int J, const Slots& s, const double* tc, cpx<T>* x, cudaStream_t st) {
  dim3 g(blocks_for(2LL * s.ns + s.nq, TPB), J);
  stokes_transform_kernel<T><<<g, TPB, 0, st>>>(dir, J, s, tc, x);
}

template <class T>
void launch_dft_forward(int K, int J, long long nblk, const double* x, cpx<T>* X, const T* cosk, const T* sink,
                        cudaStream_t st) {
  const size_t smem = ((size_t)K * DFT_COLS + 2 * (size_t)K) * sizeof(T);
  cudaFuncSetAttribute(dft_fwd_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dft_fwd_kernel<T><<<blocks_for(nblk, DFT_COLS), DFT_THREADS, smem, st>>>(K, J, nblk, x, X, cosk, sink);
}

template <class T>
void launch_dft_inverse(int K, int J, long long nblk, const cpx<T>* X, double* y, const T* cosk, const T* sink,
                        cudaStream_t st) {
  const size_t smem = (size_t)J * DFT_COLS * sizeof(cpx<T>) + 2 * (size_t)K * sizeof(T);
  cudaFuncSetAttribute(dft_inv_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dft_inv_kernel<T><<<blocks_for(nblk, DFT_COLS), DFT_THREADS, smem, st>>>(K, J, nblk, X, y, cosk, sink);
}

void launch_mask_blocks(const Slots& s, long long nvec, int ncomp, double* x, cudaStream_t st) {
  mask_kernel<<<blocks_for(nvec * s.nblk, TPB), TPB, 0, st>>>(s, nvec, ncomp, x);
}
void launch_copy_d2f(const double* a, float* b, long long n, cudaStream_t st) {
  d2f_kernel<<<blocks_for(n, TPB), TPB, 0, st>>>(a, b, n);
}
void launch_copy_f2d(const float* a, double* b, long long n, cudaStream_t st) {
  f2d_kernel<<<blocks_for(n, TPB), TPB, 0, st>>>(a, b, n);
}
void launch_count_nonfinite(const double* a, long long n, int* count, cudaStream_t st) {
  nonfinite_kernel<<<blocks_for(n, TPB), TPB, 0, st>>>(a, n, count);
}

#define PINT_INST(T)                                                                                              \
  template void launch_block_matvec<T>(const BlkArgs<T>&, cudaStream_t);                                          \
  template void launch_combo<T>(const ComboArgs<T>&, cudaStream_t);                                               \
  template void launch_bres<T>(const BResArgs<T>&, cudaStream_t);                                                 \
  template void launch_lincomb<T>(int, long long, long long, cpx<T>*, long long, const cpx<T>*, long long,        \
                                  const double*, const cpx<T>*, long long, const double*, const int*,             \
                                  cudaStream_t);                                                                  \
  template void launch_stokes_transform<T>(int, int, const Slots&, const double*, cpx<T>*, cudaStream_t);         \
  template void launch_dft_forward<T>(int, int, long long, const double*, cpx<T>*, const T*, const T*,            \
                                      cudaStream_t);                                                              \
  template void launch_dft_inverse<T>(int, int, long long, const cpx<T>*, double*, const T*, const T*,            \
                                      cudaStream_t);
PINT_INST(float)
PINT_INST(double)
#undef PINT_INST

}  // namespace pint
