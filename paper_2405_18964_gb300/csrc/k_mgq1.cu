// k_mgq1.cu -- pressure multigrid on the corner-pinned Q1 operators
// a M_p + b K_p (the K_p^{-1} of the Schur complement approximations,
// Sec. 3.2 and Sec. 4) with the level sizes fixed at compile time.
//
// The method is the one of mg_kernel<T, 1> (k_mg.cu) -- geometric multigrid
// with 4-colour SOR, colours (ix mod 2, iy mod 2) with the pinned corner
// (0, 0) left out, `pre` sweeps in colour order 0..3 and `post` sweeps in
// reverse order, the stencil in difference form, residual, restriction
// R = P^T of the bilinear interpolation, dense FP64 solve on the coarsest
// grid, prolongation P, zero initial guess, `cycles` V-cycles (Sec. 3.4:
// "geometric multigrid ... with successive over-relaxation") -- and every
// node's update is the same arithmetic in the same order.  What differs is
// where the data lives and how the work is distributed:
//  * every level is stored per colour: four sub-grids holding the nodes
//    (2a + TX, 2b + TY), each with one zero slot before position 0 in both
//    directions and zero padding after its last node, so a colour phase
//    walks one contiguous sub-grid and every neighbour lies at a
//    compile-time offset; a tap that leaves the domain reads a zero slot
//    (its weight is zero as well);
//  * the iterates and right-hand sides of every level stay in shared memory
//    for the whole solve (105 KB for 64 x 64 elements in FP32, so two CTAs
//    share an SM); the residual (one buffer that every level reuses,
//    written once and read once per level and V-cycle) lives in the job's
//    workspace, in the same layout;
//  * the interior nodes' weights are held in registers.
// One CTA owns one field for the whole solve.
#include "kernels.h"
#include "mg_weights.cuh"

namespace pint {

namespace {

constexpr int ilog2q(int v) { return v <= 1 ? 0 : 1 + ilog2q(v / 2); }
// floor(v / 2) for small v of either sign
constexpr int fl2q(int v) { return v >= 0 ? v / 2 : -((1 - v) / 2); }

// complex elements of one level of N elements per side (4 colours, each
// (N/2 + 2)^2 slots: N/2 + 1 positions plus the zero slot in front)
constexpr int qsize(int N) { return 4 * (N / 2 + 2) * (N / 2 + 2); }

template <int NF, int L>
struct QLev {
  static constexpr int N = NF >> L;      // elements per side
  static constexpr int P = N / 2 + 2;    // row pitch of a colour sub-grid
  static constexpr int SUB = P * P;      // one colour (a level: 4 SUB = qsize(N))
};

// shared-memory map (complex elements): iterates of levels 0..NL-1, right-
// hand sides of levels 1..NL-1, then the finest right-hand side
template <int NF>
constexpr int q_levels() { return ilog2q(NF); }
template <int NF>
constexpr int q_xoff(int l) {
  int o = 0;
  for (int k = 0; k < l; ++k) o += qsize(NF >> k);
  return o;
}
template <int NF>
constexpr int q_boff(int l) {
  int o = q_xoff<NF>(q_levels<NF>());
  for (int k = 1; k < l; ++k) o += qsize(NF >> k);
  return o;
}
template <int NF>
constexpr int q_roff() { return q_boff<NF>(q_levels<NF>()); }
template <int NF>
constexpr int q_elems() { return q_roff<NF>() + qsize(NF); }

// Dynamic shared memory a CTA may hold: the 227 KB of an SM less room for
// the kernel's static arrays.
constexpr long long Q1P_SMEM_BUDGET = 232448 - 4096;

template <class T>
struct QCtx {
  cpx<T>* dsm;       // shared-memory base
  cpx<T>* B0;        // finest right-hand side
  cpx<T>* R;         // residual buffer (workspace)
  const T* sw;       // [NL][9 node types][9] real weights
  const T* srs;      // [NL][9] a * (mass row sum)
  const T* sdi;      // [NL][9] inverse diagonals
  T omega;
  int pre, post;
  const double* inv;
};

template <class T, int NF, int L>
__device__ __forceinline__ cpx<T>* qx(const QCtx<T>& c) { return c.dsm + q_xoff<NF>(L); }
template <class T, int NF, int L>
__device__ __forceinline__ cpx<T>* qb(const QCtx<T>& c) {
  if constexpr (L == 0)
    return c.B0;
  else
    return c.dsm + q_boff<NF>(L);
}

// slot of node (ix, iy), -1 <= ix, iy <= N + 1, on level L
template <int NF, int L>
__device__ __forceinline__ int qslot(int ix, int iy) {
  using V = QLev<NF, L>;
  return ((ix & 1) + 2 * (iy & 1)) * V::SUB + ((iy >> 1) + 1) * V::P + (ix >> 1) + 1;
}

// (A x) at the slot idx of a node of colour (TX, TY) in difference form:
// rs x_c + sum_{k != c} w_k (x_k - x_c), taps in the order of stencil_q1d.
template <class T, int NF, int L, int TX, int TY, class WT>
__device__ __forceinline__ cpx<T> q1_stencil(const cpx<T>* x, int idx, const WT& w, T rs) {
  using V = QLev<NF, L>;
  const cpx<T> xc = x[idx];
  cpx<T> acc = rs * xc;
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      if (dx == 0 && dy == 0) continue;
      const int off = ((((TX + dx) & 1) + 2 * ((TY + dy) & 1)) - (TX + 2 * TY)) * V::SUB +
                      fl2q(TY + dy) * V::P + fl2q(TX + dx);
      rfma(acc, w[(dy + 1) * 3 + (dx + 1)], x[idx + off] - xc);
    }
  return acc;
}

// node type along one axis (0: low boundary, 1: interior, 2: high boundary)
template <int N, int TX>
__device__ __forceinline__ int axis_type(int ix) {
  if (TX == 1) return 1;
  return ix == 0 ? 0 : (ix == N ? 2 : 1);
}

// ---- one SOR colour: the nodes of sub-grid (TX, TY) ------------------------
template <class T, int NF, int L, int TX, int TY>
__device__ __forceinline__ void q1_colour(const QCtx<T>& c, cpx<T>* X, const cpx<T>* B) {
  using V = QLev<NF, L>;
  constexpr int HX = TX ? V::N / 2 : V::N / 2 + 1, HY = TY ? V::N / 2 : V::N / 2 + 1;
  constexpr int base = (TX + 2 * TY) * V::SUB + V::P + 1;
  if (threadIdx.x >= HX * HY) return;  // no node for this thread (coarse levels): straight to the barrier
  T w[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) w[k] = c.sw[(L * 9 + 4) * 9 + k];
  const T rs = c.srs[L * 9 + 4], di = c.sdi[L * 9 + 4];
  const T omega = c.omega;
  for (int q = threadIdx.x; q < HX * HY; q += blockDim.x) {
    if (TX == 0 && TY == 0 && q == 0) continue;  // pinned corner
    const int a = q % HX, b = q / HX;
    const int type = axis_type<V::N, TX>(2 * a + TX) + 3 * axis_type<V::N, TY>(2 * b + TY);
    const int idx = base + b * V::P + a;
    cpx<T> ax;
    T d;
    if (type == 4) {
      ax = q1_stencil<T, NF, L, TX, TY>(X, idx, w, rs);
      d = di;
    } else {
      const T* wb = c.sw + (L * 9 + type) * 9;
      ax = q1_stencil<T, NF, L, TX, TY>(X, idx, wb, c.srs[L * 9 + type]);
      d = c.sdi[L * 9 + type];
    }
    X[idx] = X[idx] + omega * d * (B[idx] - ax);
  }
}

template <class T, int NF, int L>
__device__ __forceinline__ void q1_sweeps(const QCtx<T>& c, cpx<T>* X, const cpx<T>* B, int count, bool down) {
  for (int s = 0; s < count; ++s)
    for (int i = 0; i < 4; ++i) {
      switch (down ? i : 3 - i) {
        case 0: q1_colour<T, NF, L, 0, 0>(c, X, B); break;
        case 1: q1_colour<T, NF, L, 1, 0>(c, X, B); break;
        case 2: q1_colour<T, NF, L, 0, 1>(c, X, B); break;
        default: q1_colour<T, NF, L, 1, 1>(c, X, B); break;
      }
      __syncthreads();
    }
}

// ---- residual r = b - A x on the nodes of colour (TX, TY) (0 at the pin) ---
template <class T, int NF, int L, int TX, int TY>
__device__ __forceinline__ void q1_residual(const QCtx<T>& c, const cpx<T>* X, const cpx<T>* B, cpx<T>* R) {
  using V = QLev<NF, L>;
  constexpr int HX = TX ? V::N / 2 : V::N / 2 + 1, HY = TY ? V::N / 2 : V::N / 2 + 1;
  constexpr int base = (TX + 2 * TY) * V::SUB + V::P + 1;
  if (threadIdx.x >= HX * HY) return;
  T w[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) w[k] = c.sw[(L * 9 + 4) * 9 + k];
  const T rs = c.srs[L * 9 + 4];
  for (int q = threadIdx.x; q < HX * HY; q += blockDim.x) {
    const int a = q % HX, b = q / HX;
    const int idx = base + b * V::P + a;
    cpx<T> r = czero<T>();
    if (!(TX == 0 && TY == 0 && q == 0)) {
      const int type = axis_type<V::N, TX>(2 * a + TX) + 3 * axis_type<V::N, TY>(2 * b + TY);
      if (type == 4)
        r = B[idx] - q1_stencil<T, NF, L, TX, TY>(X, idx, w, rs);
      else
        r = B[idx] - q1_stencil<T, NF, L, TX, TY>(X, idx, c.sw + (L * 9 + type) * 9, c.srs[L * 9 + type]);
    }
    R[idx] = r;
  }
}

// ---- restriction b_c = P^T r onto the coarse nodes of colour (TX, TY); the
// coarse iterate is zeroed on the same nodes -------------------------------
template <class T, int NF, int L, int TX, int TY>
__device__ __forceinline__ void q1_restrict(const cpx<T>* R, cpx<T>* Bc, cpx<T>* Xc) {
  using F = QLev<NF, L>;
  using C = QLev<NF, L + 1>;
  constexpr int HX = TX ? C::N / 2 : C::N / 2 + 1, HY = TY ? C::N / 2 : C::N / 2 + 1;
  constexpr int base = (TX + 2 * TY) * C::SUB + C::P + 1;
  for (int q = threadIdx.x; q < HX * HY; q += blockDim.x) {
    const int A = q % HX, Bq = q / HX;
    const int ix = 2 * A + TX, iy = 2 * Bq + TY;
    cpx<T> acc = czero<T>();
    if ((ix | iy) != 0) {
#pragma unroll
      for (int oy = -1; oy <= 1; ++oy) {
        const int fy = 2 * iy + oy;
        if (fy < 0 || fy > F::N) continue;
        const T wy = oy == 0 ? T(1) : T(0.5);
        cpx<T> s = czero<T>();
#pragma unroll
        for (int ox = -1; ox <= 1; ++ox) {
          const int fx = 2 * ix + ox;
          if (fx < 0 || fx > F::N) continue;
          rfma(s, ox == 0 ? T(1) : T(0.5), R[qslot<NF, L>(fx, fy)]);
        }
        rfma(acc, wy, s);
      }
    }
    const int idx = base + Bq * C::P + A;
    Bc[idx] = acc;
    Xc[idx] = czero<T>();
  }
}

// ---- prolongation x += P x_c on the fine nodes of colour (TX, TY) ----------
template <class T, int NF, int L, int TX, int TY>
__device__ __forceinline__ void q1_prolong(cpx<T>* X, const cpx<T>* Xc) {
  using F = QLev<NF, L>;
  using C = QLev<NF, L + 1>;
  constexpr int HX = TX ? F::N / 2 : F::N / 2 + 1, HY = TY ? F::N / 2 : F::N / 2 + 1;
  constexpr int base = (TX + 2 * TY) * F::SUB + F::P + 1;
  constexpr int nc = C::N + 1;
  for (int q = threadIdx.x; q < HX * HY; q += blockDim.x) {
    if (TX == 0 && TY == 0 && q == 0) continue;  // pinned corner
    const int a = q % HX, b = q / HX;
    const int ix = 2 * a + TX, iy = 2 * b + TY;
    const int bx = ix >> 1, by = iy >> 1;
    const T wx1 = (ix & 1) ? T(0.5) : T(0), wx0 = (ix & 1) ? T(0.5) : T(1);
    const T wy1 = (iy & 1) ? T(0.5) : T(0), wy0 = (iy & 1) ? T(0.5) : T(1);
    const int bx1 = clampi(bx + 1, 0, nc - 1), by1 = clampi(by + 1, 0, nc - 1);
    cpx<T> s0 = czero<T>(), s1 = czero<T>();
    rfma(s0, wx0, Xc[qslot<NF, L + 1>(bx, by)]);
    rfma(s0, wx1, Xc[qslot<NF, L + 1>(bx1, by)]);
    rfma(s1, wx0, Xc[qslot<NF, L + 1>(bx, by1)]);
    rfma(s1, wx1, Xc[qslot<NF, L + 1>(bx1, by1)]);
    cpx<T> acc = czero<T>();
    rfma(acc, wy0, s0);
    rfma(acc, wy1, s1);
    const int idx = base + b * F::P + a;
    X[idx] = X[idx] + acc;
  }
}

#define PINT_Q1_COLOURS(fn, ...)          \
  fn<T, NF, L, 0, 0>(__VA_ARGS__);        \
  fn<T, NF, L, 1, 0>(__VA_ARGS__);        \
  fn<T, NF, L, 0, 1>(__VA_ARGS__);        \
  fn<T, NF, L, 1, 1>(__VA_ARGS__);

// ---- one V-cycle from level L down ----------------------------------------
template <class T, int NF, int L>
__device__ void q1_vcycle(const QCtx<T>& c) {
  constexpr int NL = q_levels<NF>();
  cpx<T>* X = qx<T, NF, L>(c);
  const cpx<T>* B = qb<T, NF, L>(c);
  if constexpr (L == NL - 1) {
    // coarsest grid (2 x 2 elements, 3 x 3 nodes, 8 unknowns): dense FP64 solve
    static_assert(QLev<NF, L>::N == 2, "coarsest level has 2 elements per side");
    for (int u = threadIdx.x; u < 8; u += blockDim.x) {
      double sr = 0.0, si = 0.0;
      for (int k = 0; k < 8; ++k) {
        const int node = k + 1;
        const cpx<T> bk = B[qslot<NF, L>(node % 3, node / 3)];
        const double ir = c.inv[(u * PINT_NC_MAX + k) * 2], ii = c.inv[(u * PINT_NC_MAX + k) * 2 + 1];
        sr += ir * (double)bk.x - ii * (double)bk.y;
        si += ir * (double)bk.y + ii * (double)bk.x;
      }
      const int node = u + 1;
      X[qslot<NF, L>(node % 3, node / 3)] = mkc<T>(T(sr), T(si));
    }
    __syncthreads();
  } else {
    q1_sweeps<T, NF, L>(c, X, B, c.pre, true);
    cpx<T>* R = c.R;
    PINT_Q1_COLOURS(q1_residual, c, X, B, R)
    __syncthreads();
    cpx<T>* Xc = qx<T, NF, L + 1>(c);
    PINT_Q1_COLOURS(q1_restrict, R, qb<T, NF, L + 1>(c), Xc)
    __syncthreads();
    q1_vcycle<T, NF, L + 1>(c);
    PINT_Q1_COLOURS(q1_prolong, X, Xc)
    __syncthreads();
    q1_sweeps<T, NF, L>(c, X, B, c.post, false);
  }
}

// Up to 128 registers a thread (every tap of a node in flight): CTAs of up
// to 256 threads, two per SM (MAXT = 256), or of up to 512, one per SM.
template <class T, int NF, int MAXT>
__global__ void __launch_bounds__(MAXT, MAXT <= 256 ? 2 : 1) mg_q1p_kernel(MGLaunch<T> L) {
  constexpr int NL = q_levels<NF>();
  using V0 = QLev<NF, 0>;
  constexpr int n0 = NF + 1;
  __shared__ T s_w[NL * 81];
  __shared__ T s_rs[NL * 9];
  __shared__ T s_di[NL * 9];
  extern __shared__ __align__(16) unsigned char q1p_dsm[];
  static_assert(q_elems<NF>() >= NL * 90, "room for the complex weights");
  const FieldJob jb = L.jobs[blockIdx.x];
  if (L.active && !L.active[jb.freq]) return;
  const OpCoef oc = L.ops[jb.op];
  const cpx<double> a = mkc<double>(oc.ar, oc.ai);
  // stencil weights, mass row sums and inverse diagonals of every level
  // (FP64 -> T), real operator, all levels at once; the complex weights
  // pass through the (not yet used) dynamic shared memory
  {
    cpx<T>* tw = reinterpret_cast<cpx<T>*>(q1p_dsm);
    cpx<T>* td = tw + NL * 81;
    for (int q = threadIdx.x; q < NL * 90; q += blockDim.x) {
      const int l = q / 90, r = q - l * 90;
      const int n = (NF >> l) + 1;
      if (r < 81)
        level_weight<T, 1>(L.t64, l, n, a, oc.b, r, tw + l * 81, td + l * 9);
      else
        s_rs[l * 9 + r - 81] = level_rowsum_q1<T>(L.t64, l, n, a.x, r - 81);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < NL * 81; q += blockDim.x) s_w[q] = tw[q].x;
    for (int q = threadIdx.x; q < NL * 9; q += blockDim.x) s_di[q] = td[q].x;
    __syncthreads();
  }
  QCtx<T> c;
  c.dsm = reinterpret_cast<cpx<T>*>(q1p_dsm);
  c.B0 = c.dsm + q_roff<NF>();
  c.R = L.ws + (size_t)blockIdx.x * L.fields_per_job * L.lay.per_job;
  c.sw = s_w;
  c.srs = s_rs;
  c.sdi = s_di;
  c.omega = T(L.omega);
  c.pre = L.pre;
  c.post = L.post;
  c.inv = L.coarse_inv + (size_t)jb.op * PINT_NC_MAX * PINT_NC_MAX * 2;
  // zero iterates (zero slots and padding included) and coarse right-hand
  // sides; the finest right-hand side into the colour layout
  for (int q = threadIdx.x; q < q_roff<NF>(); q += blockDim.x) c.dsm[q] = czero<T>();
  {
    const cpx<T>* in = L.bbase + jb.b_off[0];
    for (int q = threadIdx.x; q < qsize(NF); q += blockDim.x) {
      const int col = q / V0::SUB, rem = q - col * V0::SUB;
      const int ix = 2 * (rem % V0::P - 1) + (col & 1), iy = 2 * (rem / V0::P - 1) + (col >> 1);
      cpx<T> v = czero<T>();
      if (ix >= 0 && iy >= 0 && ix <= NF && iy <= NF) v = in[(size_t)iy * n0 + ix];
      c.B0[q] = v;
    }
  }
  __syncthreads();
  for (int cyc = 0; cyc < L.cycles; ++cyc) q1_vcycle<T, NF, 0>(c);
  // result back to the natural layout (the pinned corner stays 0)
  {
    const cpx<T>* X0 = qx<T, NF, 0>(c);
    cpx<T>* out = L.xbase + jb.x_off[0];
    for (int i = threadIdx.x; i < n0 * n0; i += blockDim.x) out[i] = X0[qslot<NF, 0>(i % n0, i / n0)];
  }
}

template <class T, int NF, int MAXT>
bool q1_launch(const MGLaunch<T>& L, int threads, cudaStream_t st) {
  constexpr long long bytes = (long long)q_elems<NF>() * (long long)sizeof(cpx<T>);
  if constexpr (bytes > Q1P_SMEM_BUDGET) {
    return false;
  } else {
    if (L.lay.per_job < qsize(NF)) return false;  // workspace too small for the residual
    static const bool ok = [] {
      const cudaError_t e =
          cudaFuncSetAttribute(mg_q1p_kernel<T, NF, MAXT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      if (e != cudaSuccess) cudaGetLastError();
      return e == cudaSuccess;
    }();
    if (!ok) return false;
    mg_q1p_kernel<T, NF, MAXT><<<L.njobs, threads, (size_t)bytes, st>>>(L);
    return true;
  }
}

template <class T, int NF>
bool q1_launch_nf(const MGLaunch<T>& L, int threads, cudaStream_t st) {
  // larger thread requests are reduced to 512
  return threads <= 256 ? q1_launch<T, NF, 256>(L, threads, st) : q1_launch<T, NF, 512>(L, 512, st);
}

}  // namespace

// Launches the compile-time-sized pressure multigrid when it covers this
// launch (real Q1 operator, no convection, one field per job, finest grid of
// 4..64 elements per side whose levels fit in shared memory, 128..1024
// threads in whole warps, more than 512 reduced to 512); returns false
// (nothing launched) otherwise.
template <class T>
bool launch_mg_q1p(const MGLaunch<T>& L, int threads, cudaStream_t st) {
  if (L.space != 1 || L.conv || L.cw || L.fields_per_job != 1 || threads < 128 || threads > 1024 || threads % 32)
    return false;
  const int N = L.lay.n[0] - 1;
  if (N < 4 || L.lay.nlev != ilog2q(N) || (1 << L.lay.nlev) != N) return false;
  for (int l = 0; l < L.lay.nlev; ++l)
    if (L.lay.n[l] != (N >> l) + 1) return false;
  switch (N) {
    case 4: return q1_launch_nf<T, 4>(L, threads, st);
    case 8: return q1_launch_nf<T, 8>(L, threads, st);
    case 16: return q1_launch_nf<T, 16>(L, threads, st);
    case 32: return q1_launch_nf<T, 32>(L, threads, st);
    case 64: return q1_launch_nf<T, 64>(L, threads, st);
    default: return false;
  }
}

template bool launch_mg_q1p<float>(const MGLaunch<float>&, int, cudaStream_t);
template bool launch_mg_q1p<double>(const MGLaunch<double>&, int, cudaStream_t);

}  // namespace pint
