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
#include <atomic>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "kernels.h"
#include "mg_weights.cuh"

namespace pint {

constexpr int MG_THREADS = 256;


// (A x) at a node: sum_k w_k x_k (+ c sum_k N_k x_k for convection).
template <class T, int SP, bool CONV, bool CW>
__device__ __forceinline__ cpx<T> stencil(const cpx<T>* __restrict__ w, const T* __restrict__ nrow, T c, int n,
                                          int ix, int iy, const cpx<T>* __restrict__ x) {
  constexpr int W = SP == 2 ? 5 : 3;
  constexpr int H = W / 2;
  int cols[W];
#pragma unroll
  for (int d = 0; d < W; ++d) cols[d] = clampi(ix + d - H, 0, n - 1);
  cpx<T> acc = czero<T>(), accn = czero<T>();
#pragma unroll
  for (int dy = 0; dy < W; ++dy) {
    const cpx<T>* row = x + (size_t)clampi(iy + dy - H, 0, n - 1) * n;
#pragma unroll
    for (int dx = 0; dx < W; ++dx) {
      const cpx<T> v = row[cols[dx]];
      const cpx<T> wk = w[dy * W + dx];
      if (CW) {
        acc = acc + wk * v;
      } else {
        rfma(acc, wk.x, v);
      }
      if (CONV) rfma(accn, nrow[dy * W + dx], v);
    }
  }
  if (CONV) rfma(acc, c, accn);
  return acc;
}

// Q1 (A x) at a node from the precombined weights in difference form:
// sum_{k != c} w_k (x_k - x_c) + rs x_c, rs = a * (row sum of the mass
// stencil); the stiffness rows sum to zero exactly (Neumann rows included),
// so the near-constant mode of the pinned pressure Laplacian cancels in the
// exact differences of neighbouring values instead of in rounded sums.
template <class T>
__device__ __forceinline__ cpx<T> stencil_q1d(const cpx<T>* __restrict__ w, T rs, int n, int ix, int iy,
                                              const cpx<T>* __restrict__ x) {
  const cpx<T> xc = x[(size_t)iy * n + ix];
  cpx<T> acc = rs * xc;
#pragma unroll
  for (int dy = 0; dy < 3; ++dy) {
    const cpx<T>* row = x + (size_t)clampi(iy + dy - 1, 0, n - 1) * n;
#pragma unroll
    for (int dx = 0; dx < 3; ++dx) {
      if (dx == 1 && dy == 1) continue;
      rfma(acc, w[dy * 3 + dx].x, row[clampi(ix + dx - 1, 0, n - 1)] - xc);
    }
  }
  return acc;
}

template <int SP>
__device__ __forceinline__ bool is_unknown(int ix, int iy, int n) {
  if (SP == 2) return ix > 0 && iy > 0 && ix < n - 1 && iy < n - 1;
  return (ix | iy) != 0;
}

// One multicolour SOR colour on all fields of the job.  Q2: the colour
// (ix mod 3, iy mod 3) is walked one node-type subclass (ix mod 2, iy mod 2)
// at a time, i.e. the residue class mod 6, so that each warp's nodes share
// one weight set.  Q1: colours (ix mod 2, iy mod 2), pinned corner skipped.
template <class T, int SP, bool CONV, bool CW>
__device__ void sor_colour(int n, cpx<T>* const* X, const cpx<T>* const* B, int nf, const cpx<T>* sw,
                           const cpx<T>* sdi, const T* n2d, T c, int colour, T omega, const T* srs = nullptr) {
  if (SP == 2) {
    const int cx = colour % 3, cy = colour / 3;
    for (int sub = 0; sub < 4; ++sub) {
      const int px = sub & 1, py = sub >> 1;
      const int rx = cx + 3 * ((px + cx) & 1), ry = cy + 3 * ((py + cy) & 1);
      const int fx = rx >= 1 ? rx : 6, fy = ry >= 1 ? ry : 6;
      const int nx = fx <= n - 2 ? (n - 2 - fx) / 6 + 1 : 0;
      const int ny = fy <= n - 2 ? (n - 2 - fy) / 6 + 1 : 0;
      const int cnt = nx * ny;
      const cpx<T>* w = sw + sub * 25;
      const cpx<T> di = sdi[sub];
      for (int q = threadIdx.x; q < nf * cnt; q += blockDim.x) {
        const int f = q / cnt, r = q - f * cnt;
        const int ix = fx + 6 * (r % nx), iy = fy + 6 * (r / nx);
        const size_t id = (size_t)iy * n + ix;
        cpx<T>* x = X[f];
        const cpx<T> ax = stencil<T, SP, CONV, CW>(w, CONV ? n2d + id * 25 : nullptr, c, n, ix, iy, x);
        const cpx<T> res = B[f][id] - ax;
        x[id] = x[id] + omega * (CW ? res * di : di.x * res);
      }
    }
  } else {
    const int cx = colour & 1, cy = colour >> 1;
    const int nx = (n - 1 - cx) / 2 + 1, ny = (n - 1 - cy) / 2 + 1;
    const int cnt = nx * ny;
    for (int q = threadIdx.x; q < nf * cnt; q += blockDim.x) {
      const int f = q / cnt, r = q - f * cnt;
      const int ix = cx + 2 * (r % nx), iy = cy + 2 * (r / nx);
      if ((ix | iy) == 0) continue;
      const size_t id = (size_t)iy * n + ix;
      cpx<T>* x = X[f];
      const int type = node_type<1>(ix, iy, n);
      const cpx<T> ax = stencil_q1d<T>(sw + type * 9, srs[type], n, ix, iy, x);
      x[id] = x[id] + omega * sdi[type].x * (B[f][id] - ax);
    }
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

template <class T, int SP, bool CONV, bool CW>
__global__ void __launch_bounds__(1024, 1) mg_kernel(MGLaunch<T> L) {
  // launched for the pressure operators only (no convection); the velocity
  // multigrids, with or without convection, run in mg_q2b_kernel or the
  // compile-time-sized kernel
  static_assert(SP == 1 && !CONV && !CW, "mg_kernel serves the real pressure operators");
  __shared__ cpx<T> sw[100];
  __shared__ cpx<T> sdi[9];
  __shared__ T srs[9];
  __shared__ cpx<T>* Xs[PINT_MAXLEV][PINT_MAXF];
  __shared__ const cpx<T>* Bs[PINT_MAXLEV][PINT_MAXF];
  __shared__ cpx<T>* Rs[PINT_MAXLEV][PINT_MAXF];
  const FieldJob jb = L.jobs[blockIdx.x];
  if (L.active && !L.active[jb.freq]) return;
  const OpCoef oc = L.ops[jb.op];
  const cpx<double> a = mkc<double>(oc.ar, oc.ai);
  const double bb = oc.b;
  const T cc = T(oc.c);
  const cpx<T> ca = mkc<T>(T(oc.ar), T(oc.ai));
  const T cbT = T(oc.b);
  const T omega = T(L.omega);
  const int nf = jb.nf;
  const int nl = L.lay.nlev;
  const int last = nl - 1;
  const double* inv = L.coarse_inv + (size_t)jb.op * PINT_NC_MAX * PINT_NC_MAX * 2;
  if (threadIdx.x < PINT_MAXF) {
    const int f = threadIdx.x;
    cpx<T>* ws = L.ws + ((size_t)blockIdx.x * L.fields_per_job + (f < nf ? f : 0)) * L.lay.per_job;
    for (int l = 0; l < nl; ++l) {
      Xs[l][f] = l == 0 ? L.xbase + jb.x_off[f < nf ? f : 0] : ws + L.lay.off_x[l];
      Bs[l][f] = l == 0 ? L.bbase + jb.b_off[f < nf ? f : 0] : ws + L.lay.off_b[l];
      Rs[l][f] = ws + L.lay.off_r[l];
    }
  }
  __syncthreads();
  {
    const int n0 = L.lay.n[0];
    for (int q = threadIdx.x; q < nf * n0 * n0; q += blockDim.x) Xs[0][q / (n0 * n0)][q % (n0 * n0)] = czero<T>();
  }
  __syncthreads();

  for (int cyc = 0; cyc < L.cycles; ++cyc) {
    // ---------------- down sweep
    for (int l = 0; l < last; ++l) {
      const int n = L.lay.n[l];
      const T* n2d = CONV ? L.n2d[l] : nullptr;
      level_weights<T, SP>(L.t64, l, n, a, bb, sw, sdi);
      if (SP == 1) level_rowsums_q1<T>(L.t64, l, n, a.x, srs);
      __syncthreads();
      constexpr int NCOL = SP == 2 ? 9 : 4;
      for (int s = 0; s < L.pre; ++s)
        for (int col = 0; col < NCOL; ++col) {
          sor_colour<T, SP, CONV, CW>(n, Xs[l], Bs[l], nf, sw, sdi, n2d, cc, col, omega, srs);
          __syncthreads();
        }
      for (int q = threadIdx.x; q < nf * n * n; q += blockDim.x) {
        const int f = q / (n * n), i = q % (n * n);
        const int ix = i % n, iy = i / n;
        cpx<T> r = czero<T>();
        if (is_unknown<SP>(ix, iy, n))
          r = Bs[l][f][i] - stencil_q1d<T>(sw + node_type<1>(ix, iy, n) * 9, srs[node_type<1>(ix, iy, n)], n, ix,
                                           iy, Xs[l][f]);
        Rs[l][f][i] = r;
      }
      __syncthreads();
      const int nc = L.lay.n[l + 1];
      for (int q = threadIdx.x; q < nf * nc * nc; q += blockDim.x) {
        const int f = q / (nc * nc), i = q % (nc * nc);
        const int ix = i % nc, iy = i / nc;
        const cpx<T>* R = Rs[l][f];
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
                if (wx == T(0)) continue;
                rfma(s, wx, R[(size_t)fy * n + clampi(2 * ix + ox, 0, n - 1)]);
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
        const_cast<cpx<T>*>(Bs[l + 1][f])[i] = acc;
        Xs[l + 1][f][i] = czero<T>();
      }
      __syncthreads();
    }
    // ---------------- coarsest level: dense FP64 solve
    {
      const int n = L.lay.n[last];
      const int inner = SP == 2 ? n - 2 : n;
      const int nu = SP == 2 ? inner * inner : n * n - 1;
      for (int q = threadIdx.x; q < nf * nu; q += blockDim.x) {
        const int f = q / nu, u = q % nu;
        const cpx<T>* B = Bs[last][f];
        double sr = 0.0, si = 0.0;
        for (int k = 0; k < nu; ++k) {
          const int node = SP == 2 ? (1 + k / inner) * n + (1 + k % inner) : k + 1;
          const cpx<T> bk = B[node];
          const double ir = inv[(u * PINT_NC_MAX + k) * 2], ii = inv[(u * PINT_NC_MAX + k) * 2 + 1];
          sr += ir * (double)bk.x - ii * (double)bk.y;
          si += ir * (double)bk.y + ii * (double)bk.x;
        }
        const int node = SP == 2 ? (1 + u / inner) * n + (1 + u % inner) : u + 1;
        Xs[last][f][node] = mkc<T>(T(sr), T(si));
      }
      __syncthreads();
    }
    // ---------------- up sweep
    for (int l = last - 1; l >= 0; --l) {
      const int n = L.lay.n[l];
      const int nc = L.lay.n[l + 1];
      const T* n2d = CONV ? L.n2d[l] : nullptr;
      level_weights<T, SP>(L.t64, l, n, a, bb, sw, sdi);
      if (SP == 1) level_rowsums_q1<T>(L.t64, l, n, a.x, srs);
      for (int q = threadIdx.x; q < nf * n * n; q += blockDim.x) {
        const int f = q / (n * n), i = q % (n * n);
        const int ix = i % n, iy = i / n;
        if (!is_unknown<SP>(ix, iy, n)) continue;
        const cpx<T>* Xc = Xs[l + 1][f];
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
        Xs[l][f][i] = Xs[l][f][i] + acc;
      }
      __syncthreads();
      constexpr int NCOL = SP == 2 ? 9 : 4;
      for (int s = 0; s < L.post; ++s)
        for (int col = NCOL - 1; col >= 0; --col) {
          sor_colour<T, SP, CONV, CW>(n, Xs[l], Bs[l], nf, sw, sdi, n2d, cc, col, omega, srs);
          __syncthreads();
        }
    }
    if (last == 0) break;  // single level: the direct solve is exact
  }
}

// ============================================================================
// Q2 multigrid in a class-blocked layout.
//
// Every level of a velocity field is stored as 36 dense sub-grids of equal
// size W6 x W6 (W6 = ceil(n / 6)), one per residue class (ix mod 6,
// iy mod 6).  A colour (ix mod 3, iy mod 3) of the multicolour SOR is the
// union of four classes, which are exactly the four node types
// (vertex / midpoint in x and y).  A warp working through one class
// therefore has uniform stencil weights, couplings that are zero for its
// node type are skipped without divergence, loads coalesce, and every
// neighbour sits at a fixed offset delta[class][k] from the node (a
// per-level table in shared memory).  The input field is permuted into this
// layout at the start of a solve and the result permuted back at the end.
// ============================================================================
struct BLay {
  int w6;        // class width = ceil(n / 6)
  int s;         // class size w6 * w6
  unsigned mg;   // ceil(2^32 / w6): q / w6 == umulhi(q, mg) for the q used here
};

__host__ __device__ __forceinline__ BLay make_blay(int n) {
  BLay b;
  b.w6 = (n + 5) / 6;
  b.s = b.w6 * b.w6;
  b.mg = (unsigned)((0x100000000ull + b.w6 - 1) / b.w6);
  return b;
}
// same order as q2_blocked_index (common.cuh), with the level's sizes cached
__device__ __forceinline__ int bidx(const BLay& b, int ix, int iy) {
  return ((ix % 6) + 6 * (iy % 6)) * b.s + (iy / 6) * b.w6 + ix / 6;
}
__device__ __forceinline__ int udiv(unsigned q, unsigned mg) { return (int)__umulhi(q, mg); }

// Neighbour offsets.  A node of class (rx, ry) at sub-grid position (mx, my)
// has blocked index id = (rx + 6 ry) s + my w6 + mx; its neighbour (dx, dy)
// lies at id + xoff(rx, dx) + yoff(ry, dy) with
//   xoff = dx s + sx (1 - 6 s),   sx = [rx + dx >= 6] - [rx + dx < 0],
//   yoff = 6 dy s + sy (w6 - 36 s), sy likewise,
// i.e. the class changes by dx (wrapping mod 6) and the sub-grid column by sx.
__device__ __forceinline__ int xoff(const BLay& b, int rx, int dx) {
  const int a = rx + dx;
  const int sx = (a >= 6) - (a < 0);
  return dx * b.s + sx * (1 - 6 * b.s);
}
__device__ __forceinline__ int yoff(const BLay& b, int ry, int dy) {
  const int a = ry + dy;
  const int sy = (a >= 6) - (a < 0);
  return 6 * dy * b.s + sy * (b.w6 - 36 * b.s);
}
// Separable parts of the blocked index of node (ix, iy), ix, iy >= 0:
// bidx = xpart(ix) + ypart(iy).
__device__ __forceinline__ int xpart(const BLay& b, int ix) { return (ix % 6) * b.s + ix / 6; }
__device__ __forceinline__ int ypart(const BLay& b, int iy) { return 6 * (iy % 6) * b.s + (iy / 6) * b.w6; }

// (A x) at the node with blocked index id in class (rx, ry).
template <class T, bool CONV, bool CW>
__device__ __forceinline__ cpx<T> stencil_b(const cpx<T>* __restrict__ w, const BLay& b, const T* __restrict__ nrow,
                                            T c, int rx, int ry, int id, const cpx<T>* __restrict__ x) {
  int xo[5];
#pragma unroll
  for (int dx = -2; dx <= 2; ++dx) xo[dx + 2] = xoff(b, rx, dx);
  cpx<T> acc = czero<T>(), accn = czero<T>();
#pragma unroll
  for (int dy = -2; dy <= 2; ++dy) {
    if ((ry & 1) && (dy == -2 || dy == 2)) continue;  // midpoint rows couple to +-1 only
    const cpx<T>* row = x + id + yoff(b, ry, dy);
#pragma unroll
    for (int dx = -2; dx <= 2; ++dx) {
      if ((rx & 1) && (dx == -2 || dx == 2)) continue;
      const int k = (dy + 2) * 5 + (dx + 2);
      const cpx<T> v = row[xo[dx + 2]];
      if (CW)
        acc = acc + w[k] * v;
      else
        rfma(acc, w[k].x, v);
      if (CONV) rfma(accn, nrow[k], v);
    }
  }
  if (CONV) rfma(acc, c, accn);
  return acc;
}

template <class T, bool CONV, bool CW>
__device__ __forceinline__ void sor_node_b(int n, const BLay& b, int ccx, int ccy, int q, int& id, int& type,
                                           int& rx, int& ry, bool& valid) {
  const int sub = q / b.s, i = q - sub * b.s;
  const int my = udiv(i, b.mg), mx = i - my * b.w6;
  rx = ccx + 3 * (sub & 1);
  ry = ccy + 3 * (sub >> 1);
  const int ix = 6 * mx + rx, iy = 6 * my + ry;
  valid = q < 4 * b.s && ix >= 1 && iy >= 1 && ix <= n - 2 && iy <= n - 2;
  type = (rx & 1) + 2 * (ry & 1);
  id = (rx + 6 * ry) * b.s + i;
}

template <class T, bool CONV, bool CW>
__device__ void sor_colour_b(int n, const BLay& b, cpx<T>* X, const cpx<T>* B, const cpx<T>* sw, const cpx<T>* sdi,
                             const T* n2d, T c, int colour, T omega) {
  // the four classes of the colour (one per node type) in one parallel loop;
  // same-colour nodes do not couple, so two nodes per thread are evaluated
  // before either is written (independent loads in flight)
  const int ccx = colour % 3, ccy = colour / 3;
  const int step = blockDim.x;
  for (int q0 = threadIdx.x; q0 < 4 * b.s; q0 += 2 * step) {
    int id0, id1, t0, t1, rx0, ry0, rx1, ry1;
    bool v0, v1;
    sor_node_b<T, CONV, CW>(n, b, ccx, ccy, q0, id0, t0, rx0, ry0, v0);
    sor_node_b<T, CONV, CW>(n, b, ccx, ccy, q0 + step, id1, t1, rx1, ry1, v1);
    cpx<T> r0 = czero<T>(), r1 = czero<T>();
    if (v0)
      r0 = B[id0] - stencil_b<T, CONV, CW>(sw + t0 * 25, b, CONV ? n2d + (size_t)id0 * 25 : nullptr, c, rx0, ry0,
                                            id0, X);
    if (v1)
      r1 = B[id1] - stencil_b<T, CONV, CW>(sw + t1 * 25, b, CONV ? n2d + (size_t)id1 * 25 : nullptr, c, rx1, ry1,
                                            id1, X);
    if (v0) {
      const cpx<T> di = sdi[t0];
      X[id0] = X[id0] + omega * (CW ? r0 * di : di.x * r0);
    }
    if (v1) {
      const cpx<T> di = sdi[t1];
      X[id1] = X[id1] + omega * (CW ? r1 * di : di.x * r1);
    }
  }
}

// Class-blocked size (complex elements) of the Q2 level with n nodes per side.
__host__ __device__ __forceinline__ long long q2b_level_size(int n) {
  const long long w6 = (n + 5) / 6;
  return 36 * w6 * w6;
}

template <class T, bool CONV, bool CW>
__global__ void __launch_bounds__(1024, 1) mg_q2b_kernel(MGLaunch<T> L) {
  __shared__ cpx<T> sw[100];
  __shared__ cpx<T> sdi[9];
  // iterates of the levels in L.smem_levels live in dynamic shared memory for
  // the whole solve (each colour phase then reads its neighbours on chip);
  // right-hand sides, residuals and the other levels stay in the workspace
  extern __shared__ __align__(16) unsigned char mg_dsm[];
  const FieldJob jb = L.jobs[blockIdx.x];
  if (L.active && !L.active[jb.freq]) return;
  const OpCoef oc = L.ops[jb.op];
  const cpx<double> a = mkc<double>(oc.ar, oc.ai);
  const double bb = oc.b;
  const T cc = T(oc.c);
  const T omega = T(L.omega);
  const int nl = L.lay.nlev;
  const int last = nl - 1;
  const double* inv = L.coarse_inv + (size_t)jb.op * PINT_NC_MAX * PINT_NC_MAX * 2;
  cpx<T>* ws = L.ws + (size_t)blockIdx.x * L.fields_per_job * L.lay.per_job;
  cpx<T>* xlev[PINT_MAXLEV];
  {
    long long so = 0;
    for (int l = 0; l < nl; ++l) {
      if ((L.smem_levels >> l) & 1u) {
        xlev[l] = reinterpret_cast<cpx<T>*>(mg_dsm) + so;
        so += q2b_level_size(L.lay.n[l]);
      } else {
        xlev[l] = ws + L.lay.off_x[l];
      }
    }
  }
  auto Xl = [&](int l) { return xlev[l]; };
  auto Bl = [&](int l) { return ws + L.lay.off_b[l]; };
  auto Rl = [&](int l) { return ws + L.lay.off_r[l]; };
  const int n0 = L.lay.n[0];
  const BLay b0 = make_blay(n0);
  // permute the right-hand side into the blocked layout; zero the iterate
  // (padding slots of the blocked arrays are zeroed once here and never written)
  {
    cpx<T>* B0 = Bl(0);
    cpx<T>* X0 = Xl(0);
    for (int q = threadIdx.x; q < 36 * b0.s; q += blockDim.x) {
      B0[q] = czero<T>();
      X0[q] = czero<T>();
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n0 * n0; i += blockDim.x) {
      const int ix = i % n0, iy = i / n0;
      if (is_unknown<2>(ix, iy, n0)) B0[bidx(b0, ix, iy)] = L.bbase[jb.b_off[0] + i];
    }
  }
  __syncthreads();

  for (int cyc = 0; cyc < L.cycles; ++cyc) {
    for (int l = 0; l < last; ++l) {
      const int n = L.lay.n[l];
      const BLay b = make_blay(n);
      const T* n2d = CONV ? L.n2d[l] : nullptr;
      cpx<T>* X = Xl(l);
      const cpx<T>* B = Bl(l);
      level_weights<T, 2>(L.t64, l, n, a, bb, sw, sdi);
      __syncthreads();
      for (int s = 0; s < L.pre; ++s)
        for (int col = 0; col < 9; ++col) {
          sor_colour_b<T, CONV, CW>(n, b, X, B, sw, sdi, n2d, cc, col, omega);
          __syncthreads();
        }
      // residual over all classes (non-unknown and padding slots get 0)
      cpx<T>* R = Rl(l);
      for (int q = threadIdx.x; q < 36 * b.s; q += blockDim.x) {
        const int cls = q / b.s, i = q - cls * b.s;
        const int my = udiv(i, b.mg), mx = i - my * b.w6;
        const int id = q;
        const int rx = cls % 6, ry = cls / 6;
        const int ix = 6 * mx + rx, iy = 6 * my + ry;
        cpx<T> r = czero<T>();
        if (ix >= 1 && iy >= 1 && ix <= n - 2 && iy <= n - 2)
          r = B[id] - stencil_b<T, CONV, CW>(sw + ((rx & 1) + 2 * (ry & 1)) * 25, b,
                                             CONV ? n2d + (size_t)id * 25 : nullptr, cc, rx, ry, id, X);
        R[id] = r;
      }
      __syncthreads();
      // restriction R = P^T onto the coarse level, coarse iterate zeroed
      const int nc = L.lay.n[l + 1];
      const BLay bc = make_blay(nc);
      cpx<T>* Bc = Bl(l + 1);
      cpx<T>* Xc = Xl(l + 1);
      for (int q = threadIdx.x; q < 36 * bc.s; q += blockDim.x) {
        const int cls = q / bc.s, i = q - cls * bc.s;
        const int rx = cls % 6, ry = cls / 6;
        const int my = udiv(i, bc.mg), mx = i - my * bc.w6;
        const int ix = 6 * mx + rx, iy = 6 * my + ry;
        cpx<T> acc = czero<T>();
        if (ix >= 1 && iy >= 1 && ix <= nc - 2 && iy <= nc - 2) {
          // fine nodes 2 ix + ox, 2 iy + oy (nonzero weights: |o| <= 1, and 3 at coarse vertices)
          const int fx = 2 * ix, fy = 2 * iy;
          int xp[7], yp[7];
#pragma unroll
          for (int o = -3; o <= 3; ++o) {
            xp[o + 3] = (q2_rw(ix, o) != 0.f) ? xpart(b, fx + o) : 0;
            yp[o + 3] = (q2_rw(iy, o) != 0.f) ? ypart(b, fy + o) : 0;
          }
#pragma unroll
          for (int oy = -3; oy <= 3; ++oy) {
            const T wy = T(q2_rw(iy, oy));
            if (wy == T(0)) continue;
            cpx<T> s = czero<T>();
#pragma unroll
            for (int ox = -3; ox <= 3; ++ox) {
              const T wx = T(q2_rw(ix, ox));
              if (wx == T(0)) continue;
              rfma(s, wx, R[xp[ox + 3] + yp[oy + 3]]);
            }
            rfma(acc, wy, s);
          }
        }
        Bc[q] = acc;
        Xc[q] = czero<T>();
      }
      __syncthreads();
    }
    // coarsest level: dense FP64 solve
    {
      const int n = L.lay.n[last];
      const BLay b = make_blay(n);
      const int inner = n - 2, nu = inner * inner;
      const cpx<T>* Bc = Bl(last);
      cpx<T>* Xc = Xl(last);
      for (int u = threadIdx.x; u < nu; u += blockDim.x) {
        double sr = 0.0, si = 0.0;
        for (int k = 0; k < nu; ++k) {
          const cpx<T> bk = Bc[bidx(b, 1 + k % inner, 1 + k / inner)];
          const double ir = inv[(u * PINT_NC_MAX + k) * 2], ii = inv[(u * PINT_NC_MAX + k) * 2 + 1];
          sr += ir * (double)bk.x - ii * (double)bk.y;
          si += ir * (double)bk.y + ii * (double)bk.x;
        }
        Xc[bidx(b, 1 + u % inner, 1 + u / inner)] = mkc<T>(T(sr), T(si));
      }
      __syncthreads();
    }
    for (int l = last - 1; l >= 0; --l) {
      const int n = L.lay.n[l];
      const BLay b = make_blay(n);
      const BLay bc = make_blay(L.lay.n[l + 1]);
      const T* n2d = CONV ? L.n2d[l] : nullptr;
      cpx<T>* X = Xl(l);
      const cpx<T>* B = Bl(l);
      const cpx<T>* Xc = Xl(l + 1);
      level_weights<T, 2>(L.t64, l, n, a, bb, sw, sdi);
      // prolongation onto the fine level
      for (int q = threadIdx.x; q < 36 * b.s; q += blockDim.x) {
        const int cls = q / b.s, i = q - cls * b.s;
        const int rx = cls % 6, ry = cls / 6;
        const int my = udiv(i, b.mg), mx = i - my * b.w6;
        const int ix = 6 * mx + rx, iy = 6 * my + ry;
        if (ix < 1 || iy < 1 || ix > n - 2 || iy > n - 2) continue;
        int bx, by;
        float wx[3], wy[3];
        q2_pw(ix, bx, wx);
        q2_pw(iy, by, wy);
        int xp[3], yp[3];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
          xp[t] = wx[t] != 0.f ? xpart(bc, bx + t) : 0;
          yp[t] = wy[t] != 0.f ? ypart(bc, by + t) : 0;
        }
        cpx<T> acc = czero<T>();
#pragma unroll
        for (int ty = 0; ty < 3; ++ty) {
          if (wy[ty] == 0.f) continue;
          cpx<T> s = czero<T>();
#pragma unroll
          for (int tx = 0; tx < 3; ++tx) {
            if (wx[tx] == 0.f) continue;
            rfma(s, T(wx[tx]), Xc[xp[tx] + yp[ty]]);
          }
          rfma(acc, T(wy[ty]), s);
        }
        X[q] = X[q] + acc;
      }
      __syncthreads();
      for (int s = 0; s < L.post; ++s)
        for (int col = 8; col >= 0; --col) {
          sor_colour_b<T, CONV, CW>(n, b, X, B, sw, sdi, n2d, cc, col, omega);
          __syncthreads();
        }
    }
    if (last == 0) break;
  }
  // permute the result back to the natural layout
  {
    const cpx<T>* X0 = Xl(0);
    for (int i = threadIdx.x; i < n0 * n0; i += blockDim.x) {
      const int ix = i % n0, iy = i / n0;
      L.xbase[jb.x_off[0] + i] = is_unknown<2>(ix, iy, n0) ? X0[bidx(b0, ix, iy)] : czero<T>();
    }
  }
}

// CTA size from the number of jobs: fields are solved one per CTA, so with
// fewer jobs than SMs each job gets more threads (the kernels are compiled
// for a 64-register budget, valid for every size used here).
int cta_threads(int njobs) {
  // SM count of the device, queried once (thread-safe initialisation)
  static const int nsm = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
  }();
  if (njobs <= nsm) return 1024;
  if (njobs <= 2 * nsm) return 512;
  return MG_THREADS;
}

// ---------------------------------------------------------------------------
// Shared-memory staging of the Q2 multigrid iterates.  Levels are taken
// finest first while their class-blocked iterates fit in what a CTA may hold
// beside the kernel's static arrays (a level that does not fit is skipped
// and coarser ones are still tried).  Staging changes where the iterate
// lives, not the arithmetic: results are identical either way.
// ---------------------------------------------------------------------------
template <class T>
size_t q2_smem_budget() {
  static const size_t budget = [] {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    size_t stat = 0;
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, mg_q2b_kernel<T, true, true>) == cudaSuccess) stat = fa.sharedSizeBytes;
    cudaGetLastError();
    const size_t b = optin > (int)stat + 1024 ? (size_t)optin - stat - 1024 : 0;
    // allow every instantiation to use up to the budget (once per process)
    cudaFuncSetAttribute(mg_q2b_kernel<T, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b);
    cudaFuncSetAttribute(mg_q2b_kernel<T, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b);
    cudaFuncSetAttribute(mg_q2b_kernel<T, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b);
    cudaGetLastError();
    return b;
  }();
  return budget;
}

template <class T>
unsigned q2_smem_plan(const MGLayout& lay, size_t budget, size_t* bytes) {
  unsigned mask = 0;
  size_t tot = 0;
  for (int l = 0; l < lay.nlev; ++l) {
    const size_t sz = (size_t)q2b_level_size(lay.n[l]) * sizeof(cpx<T>);
    if (tot + sz <= budget) {
      mask |= 1u << l;
      tot += sz;
    }
  }
  *bytes = tot;
  return mask;
}

// ---------------------------------------------------------------------------
// Autotuner of the multigrid launches.  For each launch shape (space, finest
// nodes per side, job count, precision, operator variant) the launches
// after a short warm-up try every candidate -- 256, 512 and 1024 threads per
// CTA, and for velocity fields each with and without the shared-memory
// staging of the iterates -- twice each (interleaved), timed by CUDA events
// on the launch stream; every later launch of that shape uses the fastest
// on average.  The choice does not change the results: every node's update
// is the same arithmetic whichever thread performs it and wherever the
// iterate is held, and the nodes of a colour are independent.
// ---------------------------------------------------------------------------
namespace {
struct TuneCand {
  int threads;
  bool smem;
};
constexpr TuneCand TUNE_CAND[6] = {{256, false}, {512, false}, {1024, false},
                                   {256, true},  {512, true},  {1024, true}};
constexpr int TUNE_MAXC = 6;
constexpr int TUNE_WARMUP = 3;  // launches of a shape before timing (module loading, first touch)
constexpr int TUNE_REPS = 2;    // timed launches per candidate (interleaved)
constexpr int TUNE_MAXSLOTS = TUNE_MAXC * TUNE_REPS;
struct MgTune {
  int ncand = 3;  // candidates of this shape: the first ncand of TUNE_CAND
  int seen = 0;
  int best = -1;  // index into TUNE_CAND once decided
  int next = 0;   // next timing slot; slot i times candidate i % ncand
  float ms[TUNE_MAXSLOTS];
  cudaEvent_t a[TUNE_MAXSLOTS] = {}, b[TUNE_MAXSLOTS] = {};
  MgTune() {
    for (float& v : ms) v = -1.f;
  }
};
using MgKey = std::tuple<int, int, int, int, int>;  // space, n0, njobs, sizeof(T), variant
std::mutex g_tune_mu;
std::map<MgKey, MgTune> g_tune;
std::atomic<bool> g_tune_on{true};
// fixed choice used while the tuner is off: CTA threads (0 = by job count)
// and staging (-1 or 1 = the compile-time-sized kernels where they apply,
// else the general kernels staged; 2 = the same with the general kernels
// unstaged; 0 = the general kernels only, unstaged)
std::atomic<int> g_fixed_threads{0}, g_fixed_staging{-1};

// Candidate for this launch; slot >= 0 means "time this launch into slot".
// ncand: the first ncand of TUNE_CAND (2 or 3: CTA sizes only; 6: also the
// shared-memory staging).
TuneCand tune_pick(const MgKey& key, int ncand, TuneCand fallback, int& slot, cudaEvent_t& ea, cudaEvent_t& eb) {
  slot = -1;
  if (!g_tune_on.load()) return fallback;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  MgTune& t = g_tune[key];
  t.ncand = ncand;
  const int nslots = t.ncand * TUNE_REPS;
  if (t.seen < TUNE_WARMUP) {
    ++t.seen;
    return fallback;
  }
  if (t.best < 0) {
    bool all = true;
    for (int i = 0; i < nslots; ++i) {
      if (t.ms[i] < 0.f && i < t.next) {
        const cudaError_t q = cudaEventQuery(t.b[i]);
        if (q == cudaSuccess)
          cudaEventElapsedTime(&t.ms[i], t.a[i], t.b[i]);
        else if (q == cudaErrorNotReady && cudaPeekAtLastError() == cudaErrorNotReady)
          cudaGetLastError();  // "not ready" is not an error of any launch
      }
      all = all && t.ms[i] >= 0.f;
    }
    if (all) {
      float sum[TUNE_MAXC] = {};
      for (int i = 0; i < nslots; ++i) sum[i % t.ncand] += t.ms[i];
      t.best = 0;
      for (int i = 1; i < t.ncand; ++i)
        if (sum[i] < sum[t.best]) t.best = i;
      for (int i = 0; i < t.ncand; ++i) t.ms[i] = sum[i] / TUNE_REPS;  // reported: mean per candidate
      for (int i = 0; i < nslots; ++i) {
        cudaEventDestroy(t.a[i]);
        cudaEventDestroy(t.b[i]);
      }
    } else if (t.next < nslots) {
      slot = t.next++;
      cudaEventCreate(&t.a[slot]);
      cudaEventCreate(&t.b[slot]);
      ea = t.a[slot];
      eb = t.b[slot];
      return TUNE_CAND[slot % t.ncand];
    } else {
      return fallback;  // a timing is still in flight
    }
  }
  return TUNE_CAND[t.best];
}
}  // namespace

void mg_autotune_enable(bool on) { g_tune_on.store(on); }
void mg_fixed_config(int threads, int staging) {
  g_fixed_threads.store(threads);
  g_fixed_staging.store(staging);
}

std::string mg_autotune_report() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  std::string out;
  char line[512];
  for (const auto& kv : g_tune) {
    const auto& k = kv.first;
    const MgTune& t = kv.second;
    int n = snprintf(line, sizeof line, "space=%d n=%d jobs=%d %s variant=%d:", std::get<0>(k), std::get<1>(k),
                     std::get<2>(k), std::get<3>(k) == 4 ? "fp32" : "fp64", std::get<4>(k));
    for (int i = 0; i < t.ncand && n < (int)sizeof line; ++i)
      n += snprintf(line + n, sizeof line - n, " %d%s:%.3f", TUNE_CAND[i].threads, TUNE_CAND[i].smem ? "s" : "",
                    t.best >= 0 ? t.ms[i] : -1.f);
    if (n < (int)sizeof line)
      snprintf(line + n, sizeof line - n, " ms -> %d%s\n", t.best >= 0 ? TUNE_CAND[t.best].threads : 0,
               t.best >= 0 && TUNE_CAND[t.best].smem ? "s" : "");
    out += line;
  }
  return out;
}

template <class T>
void launch_mg(const MGLaunch<T>& Lin, cudaStream_t st) {
  if (Lin.njobs <= 0) return;
  MGLaunch<T> L = Lin;
  const int variant = L.conv ? 2 : (L.cw ? 1 : 0);
  int slot = -1;
  cudaEvent_t ea = nullptr, eb = nullptr;
  // the compile-time-sized kernel covers the real velocity operators W_j
  // (its own staging plan); the others run the general kernels
  // (pint_mg_launch_config with staging 0 selects the general kernels)
  const bool sized = L.space == 2 && !L.conv && !L.cw && (L.lay.n[0] - 1) / 2 >= 4 &&
                     (L.lay.n[0] - 1) / 2 <= 256 && (g_tune_on.load() || g_fixed_staging.load() != 0);
  // likewise for the real pressure operators
  const bool sized1 = L.space == 1 && !L.conv && !L.cw && L.lay.n[0] - 1 >= 4 && L.lay.n[0] - 1 <= 64 &&
                      (g_tune_on.load() || g_fixed_staging.load() != 0);
  // shared-memory staging plan of the velocity iterates (nothing for Q1)
  size_t sbytes = 0;
  const unsigned plan = L.space == 2 && !sized ? q2_smem_plan<T>(L.lay, q2_smem_budget<T>(), &sbytes) : 0u;
  const bool can_stage = plan != 0;
  // When only some frequencies are still active (late inner iterations), the
  // few live fields get larger CTAs; otherwise the tuned choice for this shape.
  const bool tail = L.active_jobs > 0 && L.active_jobs < L.njobs;
  // untuned CTA size: by job count for the general kernels; the velocity
  // kernel with compile-time level sizes 512; the pressure kernel 512 up to
  // one field per SM, else 256 (two CTAs per SM)
  auto def_threads = [&](int jobs) {
    const int t = cta_threads(jobs);
    return sized1 ? (t >= 1024 ? 512 : 256) : (sized ? 512 : t);
  };
  TuneCand pick;
  if (L.no_tune) {
    pick = TuneCand{def_threads(L.njobs), can_stage};
  } else if (!g_tune_on.load()) {
    const int ft = g_fixed_threads.load(), fs = g_fixed_staging.load();
    pick = TuneCand{ft > 0 ? ft : def_threads(tail ? L.active_jobs : L.njobs), can_stage && fs != 0 && fs != 2};
  } else if (tail) {
    pick = TuneCand{def_threads(L.active_jobs), can_stage};
  } else {
    // (the kernels with compile-time level sizes run at most 512 threads:
    // candidates 256 and 512; untuned defaults 512 for the velocity kernel,
    // 256 for the pressure kernel)
    pick = tune_pick(MgKey(L.space, L.lay.n[0], L.njobs, (int)sizeof(T), sized ? 3 : (sized1 ? 4 : variant)),
                     can_stage ? 6 : (sized || sized1 ? 2 : 3),
                     TuneCand{sized ? 512 : (sized1 ? 256 : cta_threads(L.njobs)), can_stage}, slot, ea, eb);
  }
  L.smem_levels = pick.smem ? plan : 0u;
  const size_t dyn = pick.smem ? sbytes : 0;
  dim3 grid(L.njobs), block(pick.threads);
  if (slot >= 0) cudaEventRecord(ea, st);
  if (sized && launch_mg_q2p<T>(L, pick.threads, st)) {
    // launched by the compile-time-sized kernel
  } else if (sized1 && launch_mg_q1p<T>(L, pick.threads, st)) {
    // launched by the compile-time-sized pressure kernel
  } else if (L.space == 2) {
    // one velocity field per CTA, class-blocked layout in the workspace
    if (L.conv)
      mg_q2b_kernel<T, true, true><<<grid, block, dyn, st>>>(L);
    else if (L.cw)
      mg_q2b_kernel<T, false, true><<<grid, block, dyn, st>>>(L);
    else
      mg_q2b_kernel<T, false, false><<<grid, block, dyn, st>>>(L);
  } else {
    mg_kernel<T, 1, false, false><<<grid, block, 0, st>>>(L);
  }
  if (slot >= 0) cudaEventRecord(eb, st);
}

// ---------------------------------------------------------------------------
// Jacobi-Chebyshev semi-iteration on the mass matrix (finest level), for all
// fields of a job.  Recurrence (three-term Chebyshev acceleration of the
// Jacobi iteration with D = diag(M), eigenvalues of D^{-1} M in
// [lmin, lmax]): x0 = 0, r0 = b, d0 = D^{-1} r0 / theta; x_{k+1} = x_k + d_k;
// r_{k+1} = r_k - M d_k; rho_{k+1} = 1 / (2 sigma - rho_k);
// d_{k+1} = rho_{k+1} rho_k d_k + (2 rho_{k+1} / delta) D^{-1} r_{k+1};
// theta, delta = (lmax +- lmin) / 2, sigma = theta / delta, rho_0 = 1 / sigma.
// `steps` updates of x.
// ---------------------------------------------------------------------------
template <class T, int SP>
__global__ void __launch_bounds__(1024, 1) cheb_kernel(ChebLaunch<T> L) {
  __shared__ cpx<T> sw[100];
  __shared__ cpx<T> sdi[9];
  const FieldJob jb = L.jobs[blockIdx.x];
  if (L.active && !L.active[jb.freq]) return;
  const int nf = jb.nf;
  const int n = SP == 2 ? 2 * L.tabs.N[0] + 1 : L.tabs.N[0] + 1;
  const int nn = n * n;
  level_weights<T, SP>(L.t64, 0, n, mkc<double>(1.0, 0.0), 0.0, sw, sdi);
  const double theta = 0.5 * (L.lmax + L.lmin), delta = 0.5 * (L.lmax - L.lmin);
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  auto X = [&](int f) { return L.xbase + jb.x_off[f]; };
  auto B = [&](int f) { return L.bbase + jb.b_off[f]; };
  auto Rr = [&](int f) { return L.ws + ((size_t)blockIdx.x * L.fields_per_job + f) * L.per_job; };
  __syncthreads();
  for (int q = threadIdx.x; q < nf * nn; q += blockDim.x) {
    const int f = q / nn, i = q % nn;
    const int ix = i % n, iy = i / n;
    cpx<T> ri = czero<T>(), di = czero<T>();
    if (is_unknown<SP>(ix, iy, n)) {
      const T dinv = sdi[node_type<SP>(ix, iy, n)].x;
      ri = B(f)[i];
      di = (dinv / T(theta)) * ri;
    }
    Rr(f)[i] = ri;
    Rr(f)[nn + i] = di;
    X(f)[i] = czero<T>();
  }
  __syncthreads();
  for (int k = 0; k < L.steps; ++k) {
    const bool lastk = (k == L.steps - 1);
    for (int q = threadIdx.x; q < nf * nn; q += blockDim.x) {
      const int f = q / nn, i = q % nn;
      const int ix = i % n, iy = i / n;
      if (!is_unknown<SP>(ix, iy, n)) continue;
      cpx<T>* r = Rr(f);
      const cpx<T>* d = r + nn;
      X(f)[i] = X(f)[i] + d[i];
      if (!lastk) {
        const int type = node_type<SP>(ix, iy, n);
        r[i] = r[i] - stencil<T, SP, false, false>(sw + type * (SP == 2 ? 25 : 9), nullptr, T(0), n, ix, iy, d);
      }
    }
    if (lastk) break;
    __syncthreads();
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    const T c1 = T(rho_new * rho), c2 = T(2.0 * rho_new / delta);
    for (int q = threadIdx.x; q < nf * nn; q += blockDim.x) {
      const int f = q / nn, i = q % nn;
      const int ix = i % n, iy = i / n;
      if (!is_unknown<SP>(ix, iy, n)) continue;
      cpx<T>* r = Rr(f);
      cpx<T>* d = r + nn;
      const T dinv = sdi[node_type<SP>(ix, iy, n)].x;
      cpx<T> dn = c1 * d[i];
      rfma(dn, c2 * dinv, r[i]);
      d[i] = dn;
    }
    rho = rho_new;
    __syncthreads();
  }
}

template <class T>
void launch_cheb(const ChebLaunch<T>& L, cudaStream_t st) {
  if (L.njobs <= 0) return;
  const int thr = cta_threads(L.active_jobs > 0 && L.active_jobs < L.njobs ? L.active_jobs : L.njobs);
  if (L.space == 2)
    cheb_kernel<T, 2><<<L.njobs, thr, 0, st>>>(L);
  else
    cheb_kernel<T, 1><<<L.njobs, thr, 0, st>>>(L);
}

// ---------------------------------------------------------------------------
// Per-node convection stencil tables (FP64 -> T), one level.
// ---------------------------------------------------------------------------
template <class T>
__global__ void build_n2d_kernel(Tabs<double> t64, int l, T* out, const double* __restrict__ src) {
  const int n = 2 * t64.N[l] + 1;
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)n * n * 25) return;
  const int k = (int)(q % 25);
  const long long node = q / 25;
  const int ix = (int)(node % n), iy = (int)(node / n);
  const BLay b = make_blay(n);
  double v;
  if (src) {
    v = src[q];
  } else {
    const int dx = k % 5, dy = k / 5;
    const double* tab = t64.q2[l];
    const double wx = tab[(size_t)(2 * n + ix) * 5 + dx], xx = tab[(size_t)(3 * n + ix) * 5 + dx];
    const double wy = tab[(size_t)(2 * n + iy) * 5 + dy], xy = tab[(size_t)(3 * n + iy) * 5 + dy];
    v = 2.0 * (wx * xy - xx * wy);
  }
  out[(size_t)bidx(b, ix, iy) * 25 + k] = T(v);
}

template <class T>
__global__ void build_np2d_kernel(Tabs<double> t64, T* out, const double* __restrict__ src) {
  const int n = t64.N[0] + 1;
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (long long)n * n * 9) return;
  if (src) {
    out[q] = T(src[q]);
    return;
  }
  const int k = (int)(q % 9);
  const long long node = q / 9;
  const int ix = (int)(node % n), iy = (int)(node / n);
  const int dx = k % 3, dy = k / 3;
  const double* tab = t64.q1[0];
  const double wx = tab[(size_t)(2 * n + ix) * 3 + dx], xx = tab[(size_t)(3 * n + ix) * 3 + dx];
  const double wy = tab[(size_t)(2 * n + iy) * 3 + dy], xy = tab[(size_t)(3 * n + iy) * 3 + dy];
  out[q] = T(2.0 * (wx * xy - xx * wy));
}

template <class T>
void launch_build_np2d(const Tabs<double>& t64, T* out, const double* src, cudaStream_t st) {
  const int n = t64.N[0] + 1;
  const long long tot = (long long)n * n * 9;
  build_np2d_kernel<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(t64, out, src);
}

template <class T>
void launch_build_n2d(const Tabs<double>& t64, int l, T* out, const double* src, cudaStream_t st) {
  const int n = 2 * t64.N[l] + 1;
  const long long tot = (long long)n * n * 25;
  build_n2d_kernel<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(t64, l, out, src);
}

// ---------------------------------------------------------------------------
// Coarse-grid dense inverses (one thread per operator, FP64).
// ---------------------------------------------------------------------------
__global__ void coarse_setup_kernel(Tabs<double> tabs, const OpCoef* ops, const int* op_space, const int* op_conv,
                                    int nops, double* inv, int* status, const double* conv_last) {
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
      if (sp == 2 && op_conv[op] && conv_last) {
        // general wind: the separable mass and stiffness parts plus c times
        // the node's convection stencil
        v = q2_op<double, false>(tabs.q2[last], n, ix, iy, e, a, oc.b, 0.0);
        const double* st = conv_last + (size_t)nd * 25;
        cpx<double> acc = czero<double>();
        for (int kk = 0; kk < 25; ++kk) {
          const int jx = ix + kk % 5 - 2, jy = iy + kk / 5 - 2;
          if (jx < 0 || jx >= n || jy < 0 || jy >= n) continue;
          acc = acc + st[kk] * e[jy * n + jx];
        }
        v = v + oc.c * acc;
      } else if (sp == 2)
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
                         int nops, double* inv, int* status, const double* conv_last, cudaStream_t st) {
  coarse_setup_kernel<<<(nops + 63) / 64, 64, 0, st>>>(tabs, ops, op_space, op_conv, nops, inv, status, conv_last);
}

template void launch_build_np2d<float>(const Tabs<double>&, float*, const double*, cudaStream_t);
template void launch_build_np2d<double>(const Tabs<double>&, double*, const double*, cudaStream_t);
template void launch_build_n2d<float>(const Tabs<double>&, int, float*, const double*, cudaStream_t);
template void launch_build_n2d<double>(const Tabs<double>&, int, double*, const double*, cudaStream_t);
template void launch_mg<float>(const MGLaunch<float>&, cudaStream_t);
template void launch_mg<double>(const MGLaunch<double>&, cudaStream_t);
template void launch_cheb<float>(const ChebLaunch<float>&, cudaStream_t);
template void launch_cheb<double>(const ChebLaunch<double>&, cudaStream_t);

}  // namespace pint
