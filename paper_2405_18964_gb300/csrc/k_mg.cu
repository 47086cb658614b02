// k_mg.cu -- geometric multigrid with multicolour SOR and Jacobi-Chebyshev
// semi-iteration (Sec. 3.4: "Chebyshev semi-iteration ... for mass matrices",
// "a geometric multigrid method ... with successive over-relaxation").
//
// Definition implemented (shared reading with the test oracle):
//  * levels N, N/2, ..., 2 on the same square, rediscretised operators
//    (1-D band tables per level);
//  * Q2: 9 colours (ix mod 3) + 3 (iy mod 3) over the interior nodes,
//    Q1: 4 colours (ix mod 2) + 2 (iy mod 2) over all nodes but the pinned
//    corner; same-colour nodes never share a stencil, so each colour is
//    updated in parallel; `pre` sweeps in colour order 0..last, `post`
//    sweeps in reverse order, relaxation omega;
//  * residual, restriction R = P^T, coarse correction, prolongation P =
//    exact nested interpolation (1-D weights 3/8, 3/4, -1/8 for Q2 at the
//    quarter points, 1/2 for Q1 midpoints);
//  * dense FP64 solve on the coarsest grid; zero initial guess; `cycles`
//    V-cycles.
// One CTA owns one field (job) for the whole solve, so a batched MG
// application over all frequencies and components is one launch.
#include "kernels.h"

namespace pint {

constexpr int MG_THREADS = 512;

template <int SP>
__device__ __forceinline__ int nside(int N) { return SP == 2 ? 2 * N + 1 : N + 1; }

// Colour-class geometry: first index and count along one axis.
template <int SP>
__device__ __forceinline__ void colour_axis(int n, int cc, int& first, int& count) {
  if (SP == 2) {  // interior nodes 1..n-2, stride 3
    first = (cc == 0) ? 3 : cc;
    count = (first <= n - 2) ? (n - 2 - first) / 3 + 1 : 0;
  } else {  // all nodes 0..n-1, stride 2
    first = cc;
    count = (first <= n - 1) ? (n - 1 - first) / 2 + 1 : 0;
  }
}

template <int SP>
__device__ __forceinline__ bool is_unknown(int ix, int iy, int n) {
  if (SP == 2) return ix > 0 && iy > 0 && ix < n - 1 && iy < n - 1;
  return (ix | iy) != 0;
}

template <class T, int SP, bool CONV>
__device__ __forceinline__ cpx<T> op_apply(const T* tab, int n, int ix, int iy, const cpx<T>* x, cpx<T> a, T b,
                                           T c) {
  if (SP == 2) return q2_op<T, CONV>(tab, n, ix, iy, x, a, b, c);
  return q1_op<T, CONV>(tab, n, ix, iy, x, a, b, c);
}
template <class T, int SP, bool CONV>
__device__ __forceinline__ cpx<T> op_diag(const T* tab, int n, int ix, int iy, cpx<T> a, T b, T c) {
  if (SP == 2) return q2_diag<T, CONV>(tab, n, ix, iy, a, b, c);
  return q1_diag<T, CONV>(tab, n, ix, iy, a, b, c);
}

template <class T, int SP, bool CONV>
__device__ void sor_colour(const T* tab, int n, cpx<T>* x, const cpx<T>* b, int colour, cpx<T> a, T bb, T c,
                           T omega) {
  constexpr int NC = SP == 2 ? 3 : 2;
  const int cx = colour % NC, cy = colour / NC;
  int fx, nx, fy, ny;
  colour_axis<SP>(n, cx, fx, nx);
  colour_axis<SP>(n, cy, fy, ny);
  const int tot = nx * ny;
  for (int q = threadIdx.x; q < tot; q += blockDim.x) {
    const int ix = fx + NC * (q % nx);
    const int iy = fy + NC * (q / nx);
    if (SP == 1 && (ix | iy) == 0) continue;
    const size_t id = (size_t)iy * n + ix;
    const cpx<T> ax = op_apply<T, SP, CONV>(tab, n, ix, iy, x, a, bb, c);
    const cpx<T> dg = op_diag<T, SP, CONV>(tab, n, ix, iy, a, bb, c);
    const cpx<T> upd = cdiv(b[id] - ax, dg);
    x[id] = x[id] + omega * upd;
  }
}

// 1-D restriction weights (coarse node ic <- fine nodes 2ic + o, o = -3..3)
__device__ __forceinline__ float q2_rw(int ic, int o) {
  if (ic & 1) return (o == 0) ? 1.f : ((o == 1 || o == -1) ? 0.75f : 0.f);
  if (o == 0) return 1.f;
  if (o == 1 || o == -1) return 0.375f;
  if (o == 3 || o == -3) return -0.125f;
  return 0.f;
}
// 1-D prolongation taps (fine node f <- coarse base + t, t = 0..2)
__device__ __forceinline__ void q2_pw(int f, int& base, float w[3]) {
  const int r = f & 3;
  if ((f & 1) == 0) {
    base = f >> 1;
    w[0] = 1.f;
    w[1] = 0.f;
    w[2] = 0.f;
  } else if (r == 1) {
    base = (f - 1) >> 1;
    w[0] = 0.375f;
    w[1] = 0.75f;
    w[2] = -0.125f;
  } else {
    base = (f - 3) >> 1;
    w[0] = -0.125f;
    w[1] = 0.75f;
    w[2] = 0.375f;
  }
}

template <class T, int SP, bool CONV>
__global__ void __launch_bounds__(MG_THREADS) mg_kernel(MGLaunch<T> L) {
  const FieldJob jb = L.jobs[blockIdx.x];
  if (L.active && !L.active[jb.freq]) return;
  const OpCoef oc = L.ops[jb.op];
  const cpx<T> a = mkc<T>(T(oc.ar), T(oc.ai));
  const T bb = T(oc.b), cc = T(oc.c);
  const T omega = T(L.omega);
  cpx<T>* ws = L.ws + (size_t)blockIdx.x * L.lay.per_job;
  cpx<T>* x0 = L.xbase + jb.x_off;
  const cpx<T>* b0 = L.bbase + jb.b_off;
  const int nl = L.lay.nlev;
  const int last = nl - 1;
  const double* inv = L.coarse_inv + (size_t)jb.op * PINT_NC_MAX * PINT_NC_MAX * 2;

  auto Xl = [&](int l) -> cpx<T>* { return l == 0 ? x0 : ws + L.lay.off_x[l]; };
  auto Bl = [&](int l) -> const cpx<T>* { return l == 0 ? b0 : ws + L.lay.off_b[l]; };

  {
    const int n0 = L.lay.n[0];
    for (int i = threadIdx.x; i < n0 * n0; i += blockDim.x) x0[i] = czero<T>();
  }
  __syncthreads();

  for (int cyc = 0; cyc < L.cycles; ++cyc) {
    // ---------------- down sweep
    for (int l = 0; l < last; ++l) {
      const int n = L.lay.n[l];
      const T* tab = SP == 2 ? L.tabs.q2[l] : L.tabs.q1[l];
      cpx<T>* X = Xl(l);
      const cpx<T>* B = Bl(l);
      constexpr int NCOL = SP == 2 ? 9 : 4;
      for (int s = 0; s < L.pre; ++s)
        for (int col = 0; col < NCOL; ++col) {
          sor_colour<T, SP, CONV>(tab, n, X, B, col, a, bb, cc, omega);
          __syncthreads();
        }
      cpx<T>* R = ws + L.lay.off_r[l];
      for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
        const int ix = i % n, iy = i / n;
        cpx<T> r = czero<T>();
        if (is_unknown<SP>(ix, iy, n)) r = B[i] - op_apply<T, SP, CONV>(tab, n, ix, iy, X, a, bb, cc);
        R[i] = r;
      }
      __syncthreads();
      const int nc = L.lay.n[l + 1];
      cpx<T>* Bc = ws + L.lay.off_b[l + 1];
      cpx<T>* Xc = ws + L.lay.off_x[l + 1];
      for (int i = threadIdx.x; i < nc * nc; i += blockDim.x) {
        const int ix = i % nc, iy = i / nc;
        cpx<T> acc = czero<T>();
        if (is_unknown<SP>(ix, iy, nc)) {
          if (SP == 2) {
#pragma unroll
            for (int oy = -3; oy <= 3; ++oy) {
              const T wy = T(q2_rw(iy, oy));
              if (wy == T(0)) continue;
              const int fy = clampi(2 * iy + oy, 0, n - 1);
              cpx<T> s = czero<T>();
#pragma unroll
              for (int ox = -3; ox <= 3; ++ox) {
                const T wx = T(q2_rw(ix, ox));
                const int fx = clampi(2 * ix + ox, 0, n - 1);
                rfma(s, wx, R[(size_t)fy * n + fx]);
              }
              rfma(acc, wy, s);
            }
          } else {
#pragma unroll
            for (int oy = -1; oy <= 1; ++oy) {
              const int fy = 2 * iy + oy;
              if (fy < 0 || fy > n - 1) continue;
              const T wy = oy == 0 ? T(1) : T(0.5);
              cpx<T> s = czero<T>();
#pragma unroll
              for (int ox = -1; ox <= 1; ++ox) {
                const int fx = 2 * ix + ox;
                if (fx < 0 || fx > n - 1) continue;
                rfma(s, ox == 0 ? T(1) : T(0.5), R[(size_t)fy * n + fx]);
              }
              rfma(acc, wy, s);
            }
          }
        }
        Bc[i] = acc;
        Xc[i] = czero<T>();
      }
      __syncthreads();
    }
    // ---------------- coarsest level: dense FP64 solve
    {
      const int n = L.lay.n[last];
      cpx<T>* X = Xl(last);
      const cpx<T>* B = Bl(last);
      const int inner = SP == 2 ? n - 2 : n;  // interior nodes per side (Q2) / all (Q1)
      const int nu = SP == 2 ? inner * inner : n * n - 1;
      for (int u = threadIdx.x; u < nu; u += blockDim.x) {
        double sr = 0.0, si = 0.0;
        for (int k = 0; k < nu; ++k) {
          const int node = SP == 2 ? (1 + k / inner) * n + (1 + k % inner) : k + 1;
          const cpx<T> bk = B[node];
          const double ir = inv[(u * PINT_NC_MAX + k) * 2], ii = inv[(u * PINT_NC_MAX + k) * 2 + 1];
          sr += ir * (double)bk.x - ii * (double)bk.y;
          si += ir * (double)bk.y + ii * (double)bk.x;
        }
        const int node = SP == 2 ? (1 + u / inner) * n + (1 + u % inner) : u + 1;
        X[node] = mkc<T>(T(sr), T(si));
      }
      __syncthreads();
    }
    // ---------------- up sweep
    for (int l = last - 1; l >= 0; --l) {
      const int n = L.lay.n[l];
      const int nc = L.lay.n[l + 1];
      const T* tab = SP == 2 ? L.tabs.q2[l] : L.tabs.q1[l];
      cpx<T>* X = Xl(l);
      const cpx<T>* B = Bl(l);
      const cpx<T>* Xc = ws + L.lay.off_x[l + 1];
      for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
        const int ix = i % n, iy = i / n;
        if (!is_unknown<SP>(ix, iy, n)) continue;
        cpx<T> acc = czero<T>();
        if (SP == 2) {
          int bx, by;
          float wx[3], wy[3];
          q2_pw(ix, bx, wx);
          q2_pw(iy, by, wy);
#pragma unroll
          for (int ty = 0; ty < 3; ++ty) {
            if (wy[ty] == 0.f) continue;
            const int cy = clampi(by + ty, 0, nc - 1);
            cpx<T> s = czero<T>();
#pragma unroll
            for (int tx = 0; tx < 3; ++tx) rfma(s, T(wx[tx]), Xc[(size_t)cy * nc + clampi(bx + tx, 0, nc - 1)]);
            rfma(acc, T(wy[ty]), s);
          }
        } else {
          const int bx = ix >> 1, by = iy >> 1;
          const T wx1 = (ix & 1) ? T(0.5) : T(0), wx0 = (ix & 1) ? T(0.5) : T(1);
          const T wy1 = (iy & 1) ? T(0.5) : T(0), wy0 = (iy & 1) ? T(0.5) : T(1);
          const int bx1 = clampi(bx + 1, 0, nc - 1), by1 = clampi(by + 1, 0, nc - 1);
          cpx<T> s0 = czero<T>(), s1 = czero<T>();
          rfma(s0, wx0, Xc[(size_t)by * nc + bx]);
          rfma(s0, wx1, Xc[(size_t)by * nc + bx1]);
          rfma(s1, wx0, Xc[(size_t)by1 * nc + bx]);
          rfma(s1, wx1, Xc[(size_t)by1 * nc + bx1]);
          rfma(acc, wy0, s0);
          rfma(acc, wy1, s1);
        }
        X[i] = X[i] + acc;
      }
      __syncthreads();
      constexpr int NCOL = SP == 2 ? 9 : 4;
      for (int s = 0; s < L.post; ++s)
        for (int col = NCOL - 1; col >= 0; --col) {
          sor_colour<T, SP, CONV>(tab, n, X, B, col, a, bb, cc, omega);
          __syncthreads();
        }
    }
    if (last == 0) break;  // single level: the direct solve is exact
  }
}

template <class T>
void launch_mg(const MGLaunch<T>& L, cudaStream_t st) {
  if (L.njobs <= 0) return;
  dim3 grid(L.njobs), block(MG_THREADS);
  if (L.space == 2) {
    if (L.conv)
      mg_kernel<T, 2, true><<<grid, block, 0, st>>>(L);
    else
      mg_kernel<T, 2, false><<<grid, block, 0, st>>>(L);
  } else {
    if (L.conv)
      mg_kernel<T, 1, true><<<grid, block, 0, st>>>(L);
    else
      mg_kernel<T, 1, false><<<grid, block, 0, st>>>(L);
  }
}

// ---------------------------------------------------------------------------
// Jacobi-Chebyshev semi-iteration on the mass matrix (finest level).
// Recurrence (three-term Chebyshev acceleration of the Jacobi iteration with
// D = diag(M), eigenvalues of D^{-1} M in [lmin, lmax]): x0 = 0, r0 = b,
// d0 = D^{-1} r0 / theta; x_{k+1} = x_k + d_k; r_{k+1} = r_k - M d_k;
// rho_{k+1} = 1 / (2 sigma - rho_k); d_{k+1} = rho_{k+1} rho_k d_k +
// (2 rho_{k+1} / delta) D^{-1} r_{k+1}; theta, delta = (lmax +- lmin) / 2,
// sigma = theta / delta, rho_0 = 1 / sigma.  `steps` updates of x.
// ---------------------------------------------------------------------------
template <class T, int SP>
__global__ void __launch_bounds__(MG_THREADS) cheb_kernel(ChebLaunch<T> L) {
  const FieldJob jb = L.jobs[blockIdx.x];
  if (L.active && !L.active[jb.freq]) return;
  const int n = SP == 2 ? 2 * L.tabs.N[0] + 1 : L.tabs.N[0] + 1;
  const T* tab = SP == 2 ? L.tabs.q2[0] : L.tabs.q1[0];
  cpx<T>* x = L.xbase + jb.x_off;
  const cpx<T>* b = L.bbase + jb.b_off;
  cpx<T>* r = L.ws + (size_t)blockIdx.x * L.per_job;
  cpx<T>* d = r + (size_t)n * n;
  const double theta = 0.5 * (L.lmax + L.lmin), delta = 0.5 * (L.lmax - L.lmin);
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  const cpx<T> one = mkc<T>(T(1), T(0));
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    const int ix = i % n, iy = i / n;
    cpx<T> ri = czero<T>(), di = czero<T>();
    if (is_unknown<SP>(ix, iy, n)) {
      const T dg = op_diag<T, SP, false>(tab, n, ix, iy, one, T(0), T(0)).x;
      ri = b[i];
      di = (T(1) / (dg * T(theta))) * ri;
    }
    r[i] = ri;
    d[i] = di;
    x[i] = czero<T>();
  }
  __syncthreads();
  for (int k = 0; k < L.steps; ++k) {
    const bool lastk = (k == L.steps - 1);
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
      const int ix = i % n, iy = i / n;
      if (!is_unknown<SP>(ix, iy, n)) continue;
      x[i] = x[i] + d[i];
      if (!lastk) r[i] = r[i] - op_apply<T, SP, false>(tab, n, ix, iy, d, one, T(0), T(0));
    }
    if (lastk) break;
    __syncthreads();
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    const T c1 = T(rho_new * rho), c2 = T(2.0 * rho_new / delta);
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
      const int ix = i % n, iy = i / n;
      if (!is_unknown<SP>(ix, iy, n)) continue;
      const T dg = op_diag<T, SP, false>(tab, n, ix, iy, one, T(0), T(0)).x;
      cpx<T> dn = c1 * d[i];
      rfma(dn, c2 / dg, r[i]);
      d[i] = dn;
    }
    rho = rho_new;
    __syncthreads();
  }
}

template <class T>
void launch_cheb(const ChebLaunch<T>& L, cudaStream_t st) {
  if (L.njobs <= 0) return;
  if (L.space == 2)
    cheb_kernel<T, 2><<<L.njobs, MG_THREADS, 0, st>>>(L);
  else
    cheb_kernel<T, 1><<<L.njobs, MG_THREADS, 0, st>>>(L);
}

// ---------------------------------------------------------------------------
// Coarse-grid dense inverses (one thread per operator, FP64).
// ---------------------------------------------------------------------------
__global__ void coarse_setup_kernel(Tabs<double> tabs, const OpCoef* ops, const int* op_space, const int* op_conv,
                                    int nops, double* inv, int* status) {
  const int op = blockIdx.x * blockDim.x + threadIdx.x;
  if (op >= nops) return;
  const int sp = op_space[op];
  if (sp == 0) return;  // not a multigrid operator
  const int last = tabs.nlev - 1;
  const int N = tabs.N[last];
  const int n = sp == 2 ? 2 * N + 1 : N + 1;
  const int inner = sp == 2 ? n - 2 : n;
  const int nu = sp == 2 ? inner * inner : n * n - 1;
  double* out = inv + (size_t)op * PINT_NC_MAX * PINT_NC_MAX * 2;
  if (nu > PINT_NC_MAX || n * n > 25) {
    status[op] = 2;
    return;
  }
  const OpCoef oc = ops[op];
  const cpx<double> a = mkc<double>(oc.ar, oc.ai);
  cpx<double> e[25];
  cpx<double> A[PINT_NC_MAX][PINT_NC_MAX], Inv[PINT_NC_MAX][PINT_NC_MAX];
  auto node_of = [&](int u) { return sp == 2 ? (1 + u / inner) * n + (1 + u % inner) : u + 1; };
  for (int k = 0; k < nu; ++k) {
    for (int i = 0; i < n * n; ++i) e[i] = czero<double>();
    e[node_of(k)] = mkc<double>(1.0, 0.0);
    for (int u = 0; u < nu; ++u) {
      const int nd = node_of(u);
      const int ix = nd % n, iy = nd / n;
      cpx<double> v;
      if (sp == 2)
        v = op_conv[op] ? q2_op<double, true>(tabs.q2[last], n, ix, iy, e, a, oc.b, oc.c)
                        : q2_op<double, false>(tabs.q2[last], n, ix, iy, e, a, oc.b, oc.c);
      else
        v = op_conv[op] ? q1_op<double, true>(tabs.q1[last], n, ix, iy, e, a, oc.b, oc.c)
                        : q1_op<double, false>(tabs.q1[last], n, ix, iy, e, a, oc.b, oc.c);
      A[u][k] = v;
    }
  }
  for (int i = 0; i < nu; ++i)
    for (int k = 0; k < nu; ++k) Inv[i][k] = mkc<double>(i == k ? 1.0 : 0.0, 0.0);
  // Gauss-Jordan elimination with partial pivoting
  for (int col = 0; col < nu; ++col) {
    int piv = col;
    double best = -1.0;
    for (int r = col; r < nu; ++r) {
      const double m = A[r][col].x * A[r][col].x + A[r][col].y * A[r][col].y;
      if (m > best) {
        best = m;
        piv = r;
      }
    }
    if (best <= 0.0) {
      status[op] = 1;
      return;
    }
    if (piv != col)
      for (int k = 0; k < nu; ++k) {
        cpx<double> t = A[col][k];
        A[col][k] = A[piv][k];
        A[piv][k] = t;
        t = Inv[col][k];
        Inv[col][k] = Inv[piv][k];
        Inv[piv][k] = t;
      }
    const cpx<double> p = A[col][col];
    for (int k = 0; k < nu; ++k) {
      A[col][k] = cdiv(A[col][k], p);
      Inv[col][k] = cdiv(Inv[col][k], p);
    }
    for (int r = 0; r < nu; ++r) {
      if (r == col) continue;
      const cpx<double> f = A[r][col];
      for (int k = 0; k < nu; ++k) {
        A[r][k] = A[r][k] - f * A[col][k];
        Inv[r][k] = Inv[r][k] - f * Inv[col][k];
      }
    }
  }
  for (int i = 0; i < nu; ++i)
    for (int k = 0; k < nu; ++k) {
      out[(i * PINT_NC_MAX + k) * 2] = Inv[i][k].x;
      out[(i * PINT_NC_MAX + k) * 2 + 1] = Inv[i][k].y;
    }
  status[op] = 0;
}

void launch_coarse_setup(const Tabs<double>& tabs, const OpCoef* ops, const int* op_space, const int* op_conv,
                         int nops, double* inv, int* status, cudaStream_t st) {
  coarse_setup_kernel<<<(nops + 63) / 64, 64, 0, st>>>(tabs, ops, op_space, op_conv, nops, inv, status);
}

template void launch_mg<float>(const MGLaunch<float>&, cudaStream_t);
template void launch_mg<double>(const MGLaunch<double>&, cudaStream_t);
template void launch_cheb<float>(const ChebLaunch<float>&, cudaStream_t);
template void launch_cheb<double>(const ChebLaunch<double>&, cudaStream_t);

}  // namespace pint
