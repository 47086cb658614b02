// k_mgp.cu -- velocity multigrid on W_j = (1 + c1) M + c2 nu K (Stokes,
// Sec. 3.2) with the level sizes fixed at compile time.
//
// The method is the one of mg_q2b_kernel (k_mg.cu) -- geometric multigrid
// with multicolour SOR, 9 colours (ix mod 3) + 3 (iy mod 3), `pre` sweeps in
// colour order 0..8 and `post` sweeps in reverse order, residual,
// restriction R = P^T, dense FP64 solve on the coarsest grid, prolongation P
// (exact nested interpolation), zero initial guess, `cycles` V-cycles
// (Sec. 3.4: "geometric multigrid ... with successive over-relaxation") --
// and every node's update is the same arithmetic in the same order.  What
// differs is the data layout and the distribution of the work:
//  * each level's size is a template parameter, so every stencil tap is a
//    load at a compile-time offset from the node's own slot;
//  * iterates and residuals are stored per node type (ix mod 2, iy mod 2:
//    vertex or midpoint in x and y), each type an (N+1) x (N+1) sub-grid
//    ("parity layout"), which makes a neighbour's offset depend on the node
//    type only;
//  * each quarter of the CTA's warps owns one node type, so a warp's taps are
//    uniform (no skipped couplings, no divergence); a colour of one type is
//    every third node of the sub-grid in x and y, which keeps 8-byte shared
//    loads free of bank conflicts;
//  * right-hand sides are stored per residue class (ix mod 6, iy mod 6) =
//    (colour, type), so a colour phase reads them contiguously;
//  * the iterates of every level that fits stay in shared memory for the
//    whole solve (levels finest first; for 64 x 64 elements in FP32 all of
//    them), the right-hand sides and residuals in the job's workspace.
// One CTA owns one field for the whole solve.
#include "kernels.h"
#include "mg_weights.cuh"

namespace pint {

namespace {

constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v / 2); }
// floor(v / 2) for small v of either sign
constexpr int fl2(int v) { return v >= 0 ? v / 2 : -((1 - v) / 2); }

template <int NF, int L>
struct PLev {
  static constexpr int N = NF >> L;          // elements per side
  static constexpr int PX = q2p_pitch(N);    // iterate sub-grid pitch (bank-conflict free colours)
  static constexpr int PR = N + 1;           // residual sub-grid pitch
  static constexpr int SUBX = PX * (N + 1);  // one node type of the iterate
  static constexpr int SUBR = PR * (N + 1);  // one node type of the residual
  static constexpr int SIZEX = 4 * SUBX;
  static constexpr int W3 = (N + 3) / 3;     // ceil((N + 1) / 3): one residue class per side
  static constexpr int CS = W3 * W3;         // one residue class
};

// Shared-memory plan: the iterates of the levels that fit are kept on chip
// (bit l of MASKX), finest first; then the right-hand sides of the coarse
// levels (bit l of MASKB), coarsest first, whose phases are too short to hide
// a trip to L2.
constexpr long long xbytes(int N, int cbytes) { return 4LL * (N + 1) * q2p_pitch(N) * cbytes; }
constexpr long long bbytes(int N, int cbytes) { return 36LL * ((N + 3) / 3) * ((N + 3) / 3) * cbytes; }
constexpr unsigned plan_xmask(int NF, int cbytes, long long budget) {
  unsigned m = 0;
  long long tot = 0;
  for (int l = 0; (NF >> l) >= 2; ++l) {
    const long long sz = xbytes(NF >> l, cbytes);
    if (tot + sz <= budget) {
      m |= 1u << l;
      tot += sz;
    }
  }
  return m;
}
constexpr long long xtotal(int NF, int cbytes, unsigned m, int upto) {
  long long tot = 0;
  for (int l = 0; l < upto; ++l)
    if ((m >> l) & 1u) tot += xbytes(NF >> l, cbytes);
  return tot;
}
constexpr unsigned plan_bmask(int NF, int cbytes, long long budget, long long used) {
  unsigned m = 0;
  long long tot = used;
  int nl = 0;
  while ((NF >> nl) >= 2) ++nl;
  for (int l = nl - 1; l >= 1; --l) {
    const long long sz = bbytes(NF >> l, cbytes);
    if (tot + sz > budget) break;
    m |= 1u << l;
    tot += sz;
  }
  return m;
}
// offset of level `upto`'s right-hand side after all staged iterates
constexpr long long boffset(int NF, int cbytes, unsigned mx, unsigned mb, int nl, int upto) {
  long long tot = xtotal(NF, cbytes, mx, nl);
  for (int l = nl - 1; l > upto; --l)
    if ((mb >> l) & 1u) tot += bbytes(NF >> l, cbytes);
  return tot;
}

// Dynamic shared memory a CTA may hold: the 227 KB of an SM less room for
// the kernel's static arrays (weights of every level).
constexpr long long MGP_SMEM_BUDGET = 232448 - 8192 - 1024;

template <class T, int NF>
struct PPlan {
  static constexpr int NL = ilog2c(NF);
  static constexpr int CB = (int)sizeof(cpx<T>);
  static constexpr unsigned MASK = plan_xmask(NF, CB, MGP_SMEM_BUDGET);
  static constexpr long long XBYTES = xtotal(NF, CB, MASK, NL);
  static constexpr unsigned MASKB = plan_bmask(NF, CB, MGP_SMEM_BUDGET, XBYTES);
  static constexpr long long BYTES = boffset(NF, CB, MASK, MASKB, NL, 0);
};

// acc += s * v (real s, complex v): one packed FMA for FP32, two for FP64;
// each component is fma(s, v, acc) either way.
__device__ __forceinline__ void pfma(cpx<float>& acc, float s, cpx<float> v) {
  const float2 r = __ffma2_rn(make_float2(s, s), make_float2(v.x, v.y), make_float2(acc.x, acc.y));
  acc.x = r.x;
  acc.y = r.y;
}
__device__ __forceinline__ void pfma(cpx<double>& acc, double s, cpx<double> v) { rfma(acc, s, v); }

__device__ __forceinline__ void cta_bar() { __syncthreads(); }

template <class T, int NF>
struct Ctx {
  cpx<T>* X[PINT_MAXLEV];  // iterates of the levels the plan leaves in the workspace
  cpx<T>* B[PINT_MAXLEV];  // right-hand sides (class layout)
  cpx<T>* R[PINT_MAXLEV];  // residuals (per-type layout, pitch N + 1)
  const T* sw;             // [NL][4][25] real weights of W_j per level and node type
  const T* sdi;            // [NL][4] inverse diagonals
  T omega;
  int pre, post;
  int g, t, nt;            // node type of this thread's warp group, index in the group, group size
  const double* inv;
};

// Warp groups: a quarter of the CTA's warps per node type.  A colour phase
// holds the same number of nodes of each type, and a thread's nodes are
// processed one after another, each waiting for its right-hand side from L2
// when that level's is not staged; equal groups give every group the same
// number of such rounds (groups sized by coupling count, 3/8, 1/4, 1/4, 1/8,
// left the 9-coupling nodes' group with twice the rounds of the others).
__device__ __forceinline__ void type_group(int& g, int& t, int& nt) {
  const int W = blockDim.x >> 5, w = threadIdx.x >> 5;
  const int per = W >> 2;
  g = w / per;
  t = threadIdx.x - 32 * per * g;
  nt = 32 * per;
}

// ---- level pointers: shared memory where the plan keeps the iterate -------
template <class T, int NF, int L>
__device__ __forceinline__ cpx<T>* xlev(const Ctx<T, NF>& c, unsigned char* dsm) {
  using PL = PPlan<T, NF>;
  if constexpr (((PL::MASK >> L) & 1u) != 0)
    return reinterpret_cast<cpx<T>*>(dsm + xtotal(NF, PL::CB, PL::MASK, L));
  else
    return c.X[L];
}
template <class T, int NF, int L>
__device__ __forceinline__ cpx<T>* blev(const Ctx<T, NF>& c, unsigned char* dsm) {
  using PL = PPlan<T, NF>;
  if constexpr (((PL::MASKB >> L) & 1u) != 0)
    return reinterpret_cast<cpx<T>*>(dsm + boffset(NF, PL::CB, PL::MASK, PL::MASKB, PL::NL, L));
  else
    return c.B[L];
}

template <int NF, int L, int TX, int TY>
__device__ __forceinline__ int xindex(int a, int b) {
  using V = PLev<NF, L>;
  return (TX + 2 * TY) * V::SUBX + b * V::PX + a;
}

// ---- stencil of W_j at the iterate slot idx of a node of type (TX, TY) -----
// w: the type's 25 weights (registers), k = (dy + 2) * 5 + (dx + 2).
template <class T, int NF, int L, int TX, int TY>
__device__ __forceinline__ cpx<T> stencil_p(const cpx<T>* __restrict__ x, int idx, const T (&w)[25]) {
  using V = PLev<NF, L>;
  cpx<T> acc = czero<T>();
#pragma unroll
  for (int dy = -2; dy <= 2; ++dy) {
    if (TY == 1 && (dy == -2 || dy == 2)) continue;  // midpoint rows couple to +-1 only
#pragma unroll
    for (int dx = -2; dx <= 2; ++dx) {
      if (TX == 1 && (dx == -2 || dx == 2)) continue;
      constexpr int self = TX + 2 * TY;
      const int nt = ((TX + dx) & 1) + 2 * ((TY + dy) & 1);
      const int off = (nt - self) * V::SUBX + fl2(TY + dy) * V::PX + fl2(TX + dx);
      pfma(acc, w[(dy + 2) * 5 + (dx + 2)], x[idx + off]);
    }
  }
  return acc;
}

template <class T, int L, int TX, int TY>
__device__ __forceinline__ void load_weights(const T* sw, T (&w)[25]) {
  const T* src = sw + (L * 4 + TX + 2 * TY) * 25;
#pragma unroll
  for (int dy = -2; dy <= 2; ++dy)
#pragma unroll
    for (int dx = -2; dx <= 2; ++dx) {
      const int k = (dy + 2) * 5 + (dx + 2);
      const bool used = !(TY == 1 && (dy == -2 || dy == 2)) && !(TX == 1 && (dx == -2 || dx == 2));
      w[k] = used ? src[k] : T(0);
    }
}

// right-hand side slot of sub-grid position (a, b) of type (TX, TY)
template <int NF, int L, int TX, int TY>
__device__ __forceinline__ int cls_index(int a, int b) {
  using V = PLev<NF, L>;
  return ((TX + 2 * TY) * 9 + a % 3 + 3 * (b % 3)) * V::CS + (b / 3) * V::W3 + a / 3;
}

template <int NF, int L, int TX>
__device__ __forceinline__ bool interior1(int a) {
  // vertex rows: ix = 2a in [2, 2N - 2]; midpoint rows: ix = 2a + 1 in [1, 2N - 1]
  return a >= (TX == 0 ? 1 : 0) && a <= PLev<NF, L>::N - 1;
}

// ---- one colour of multicolour SOR, nodes of type (TX, TY) -----------------
template <class T, int NF, int L, int TX, int TY>
__device__ __forceinline__ void sor_colour_p(cpx<T>* X, const cpx<T>* __restrict__ B, const T (&w)[25], T di,
                                             T omega, int col, int t, int nt) {
  using V = PLev<NF, L>;
  const int cx = col % 3, cy = col / 3;
  const int ra = (2 * cx + TX) % 3, rb = (2 * cy + TY) % 3;  // a = 2^-1 (ix - TX) mod 3
  const cpx<T>* Bc = B + ((TX + 2 * TY) * 9 + ra + 3 * rb) * V::CS;
#pragma unroll 2
  for (int k = t; k < V::CS; k += nt) {
    const int a = ra + 3 * (k % V::W3), b = rb + 3 * (k / V::W3);
    if (!interior1<NF, L, TX>(a) || !interior1<NF, L, TY>(b)) continue;
    const cpx<T> bk = Bc[k];
    const int idx = xindex<NF, L, TX, TY>(a, b);
    const cpx<T> ax = stencil_p<T, NF, L, TX, TY>(X, idx, w);
    const cpx<T> r = bk - ax;
    X[idx] = X[idx] + omega * (di * r);
  }
}

template <class T, int NF, int L, int TX, int TY>
__device__ __forceinline__ void sweeps_type(const Ctx<T, NF>& c, cpx<T>* X, const cpx<T>* B, int count, bool down) {
  T w[25];
  load_weights<T, L, TX, TY>(c.sw, w);
  const T di = c.sdi[L * 4 + TX + 2 * TY];
  for (int s = 0; s < count; ++s)
    for (int i = 0; i < 9; ++i) {
      sor_colour_p<T, NF, L, TX, TY>(X, B, w, di, c.omega, down ? i : 8 - i, c.t, c.nt);
      cta_bar();
    }
}

// ---- residual r = b - W x on the nodes of type (TX, TY) (0 elsewhere) ------
// Nodes are taken in the order of their right-hand sides (contiguous reads);
// the residual goes to the per-type layout the restriction reads.
template <class T, int NF, int L, int TX, int TY>
__device__ __forceinline__ void residual_type(const Ctx<T, NF>& c, const cpx<T>* X, const cpx<T>* __restrict__ B,
                                              cpx<T>* R) {
  using V = PLev<NF, L>;
  T w[25];
  load_weights<T, L, TX, TY>(c.sw, w);
  const cpx<T>* Bt = B + (TX + 2 * TY) * 9 * V::CS;
#pragma unroll 2
  for (int q = c.t; q < 9 * V::CS; q += c.nt) {
    const int cls = q / V::CS, kk = q - cls * V::CS;
    const int a = cls % 3 + 3 * (kk % V::W3), b = cls / 3 + 3 * (kk / V::W3);
    if (a > V::N || b > V::N) continue;  // padding slot of the class layout
    cpx<T> r = czero<T>();
    if (interior1<NF, L, TX>(a) && interior1<NF, L, TY>(b))
      r = Bt[q] - stencil_p<T, NF, L, TX, TY>(X, xindex<NF, L, TX, TY>(a, b), w);
    R[(TX + 2 * TY) * V::SUBR + b * V::PR + a] = r;
  }
}

// 1-D restriction weight of fine offset o at a coarse node of type TC
template <int TC>
__device__ __forceinline__ constexpr float rw1(int o) {
  if (TC == 1) return o == 0 ? 1.f : ((o == 1 || o == -1) ? 0.75f : 0.f);
  if (o == 0) return 1.f;
  if (o == 1 || o == -1) return 0.375f;
  if (o == 3 || o == -3) return -0.125f;
  return 0.f;
}

// ---- restriction b_c = P^T r onto coarse nodes of type (TX, TY) ------------
// Coarse nodes are taken in sub-grid order, so a warp reads fine residuals
// two slots apart; their right-hand sides are written to the class layout.
template <class T, int NF, int L, int TX, int TY>
__device__ __forceinline__ void restrict_type(const Ctx<T, NF>& c, const cpx<T>* __restrict__ R, cpx<T>* Bc) {
  using F = PLev<NF, L>;
  using C = PLev<NF, L + 1>;
#pragma unroll 2
  for (int q = c.t; q < C::SUBR; q += c.nt) {
    const int A = q % C::PR, Bq = q / C::PR;
    cpx<T> acc = czero<T>();
    if (interior1<NF, L + 1, TX>(A) && interior1<NF, L + 1, TY>(Bq)) {
      // fine node 2 I + o of coarse node I = 2 A + TX: type o mod 2, position 2 A + TX + floor(o / 2)
      const int base = 2 * Bq * F::PR + 2 * A;
#pragma unroll
      for (int oy = -3; oy <= 3; ++oy) {
        const T wy = T(rw1<TY>(oy));
        if (wy == T(0)) continue;
        cpx<T> s = czero<T>();
#pragma unroll
        for (int ox = -3; ox <= 3; ++ox) {
          const T wx = T(rw1<TX>(ox));
          if (wx == T(0)) continue;
          const int ft = (ox & 1) + 2 * (oy & 1);
          const int off = ft * F::SUBR + (TY + fl2(oy)) * F::PR + (TX + fl2(ox));
          pfma(s, wx, R[base + off]);
        }
        pfma(acc, wy, s);
      }
    }
    Bc[cls_index<NF, L + 1, TX, TY>(A, Bq)] = acc;
  }
}

// ---- prolongation x += P x_c on the fine nodes of type (TX, TY) -----------
template <int TF>
__device__ __forceinline__ int prol_taps(int a, int* ct, int* cp, float* w) {
  if (TF == 0) {  // fine vertex ix = 2a: coarse node a
    ct[0] = a & 1;
    cp[0] = a >> 1;
    w[0] = 1.f;
    return 1;
  }
  // fine midpoint ix = 2a + 1 = 4 q + 1 (a even) or 4 q + 3 (a odd): coarse 2q, 2q + 1, 2q + 2
  const int q = a >> 1;
  ct[0] = 0;
  cp[0] = q;
  ct[1] = 1;
  cp[1] = q;
  ct[2] = 0;
  cp[2] = q + 1;
  w[0] = (a & 1) ? -0.125f : 0.375f;
  w[1] = 0.75f;
  w[2] = (a & 1) ? 0.375f : -0.125f;
  return 3;
}

template <class T, int NF, int L, int TX, int TY>
__device__ __forceinline__ void prolong_type(const Ctx<T, NF>& c, cpx<T>* X, const cpx<T>* __restrict__ Xc) {
  using F = PLev<NF, L>;
  using C = PLev<NF, L + 1>;
  for (int q = c.t; q < F::SUBR; q += c.nt) {
    const int a = q % F::PR, b = q / F::PR;
    if (!interior1<NF, L, TX>(a) || !interior1<NF, L, TY>(b)) continue;
    int ctx[3], cpx_[3], cty[3], cpy[3];
    float wx[3], wy[3];
    const int nx = prol_taps<TX>(a, ctx, cpx_, wx);
    const int ny = prol_taps<TY>(b, cty, cpy, wy);
    cpx<T> acc = czero<T>();
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      if (j >= ny) break;
      cpx<T> s = czero<T>();
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        if (i >= nx) break;
        pfma(s, T(wx[i]), Xc[(ctx[i] + 2 * cty[j]) * C::SUBX + cpy[j] * C::PX + cpx_[i]]);
      }
      pfma(acc, T(wy[j]), s);
    }
    const int idx = xindex<NF, L, TX, TY>(a, b);
    X[idx] = X[idx] + acc;
  }
}

#define PINT_MGP_DISPATCH(fn, ...)                     \
  switch (c.g) {                                       \
    case 0: fn<T, NF, L, 0, 0>(__VA_ARGS__); break;    \
    case 1: fn<T, NF, L, 1, 0>(__VA_ARGS__); break;    \
    case 2: fn<T, NF, L, 0, 1>(__VA_ARGS__); break;    \
    default: fn<T, NF, L, 1, 1>(__VA_ARGS__); break;   \
  }

template <class T, int NF, int L>
__device__ __forceinline__ void sweeps(const Ctx<T, NF>& c, cpx<T>* X, const cpx<T>* B, int count, bool down) {
  PINT_MGP_DISPATCH(sweeps_type, c, X, B, count, down)
}

// ---- one V-cycle from level L down ----------------------------------------
template <class T, int NF, int L>
__device__ void vcycle(const Ctx<T, NF>& c, unsigned char* dsm) {
  using V = PLev<NF, L>;
  constexpr int NL = ilog2c(NF);
  cpx<T>* X = xlev<T, NF, L>(c, dsm);
  const cpx<T>* B = blev<T, NF, L>(c, dsm);
  if constexpr (L == NL - 1) {
    // coarsest grid (2 x 2 elements, 3 x 3 unknowns): dense FP64 solve
    static_assert(V::N == 2, "coarsest level has 2 elements per side");
    for (int u = threadIdx.x; u < 9; u += blockDim.x) {
      double sr = 0.0, si = 0.0;
      for (int k = 0; k < 9; ++k) {
        const int ix = 1 + k % 3, iy = 1 + k / 3;
        const int a = ix >> 1, b = iy >> 1;
        const int tyk = (ix & 1) + 2 * (iy & 1);
        const cpx<T> bk = B[(tyk * 9 + a % 3 + 3 * (b % 3)) * V::CS + (b / 3) * V::W3 + a / 3];
        const double ir = c.inv[(u * PINT_NC_MAX + k) * 2], ii = c.inv[(u * PINT_NC_MAX + k) * 2 + 1];
        sr += ir * (double)bk.x - ii * (double)bk.y;
        si += ir * (double)bk.y + ii * (double)bk.x;
      }
      const int ix = 1 + u % 3, iy = 1 + u / 3;
      X[((ix & 1) + 2 * (iy & 1)) * V::SUBX + (iy >> 1) * V::PX + (ix >> 1)] = mkc<T>(T(sr), T(si));
    }
    cta_bar();
  } else {
    using C = PLev<NF, L + 1>;
    sweeps<T, NF, L>(c, X, B, c.pre, true);
    cpx<T>* R = c.R[L];
    PINT_MGP_DISPATCH(residual_type, c, X, B, R)
    cta_bar();
    cpx<T>* Xc = xlev<T, NF, L + 1>(c, dsm);
    PINT_MGP_DISPATCH(restrict_type, c, R, blev<T, NF, L + 1>(c, dsm))
    for (int q = threadIdx.x; q < C::SIZEX; q += blockDim.x) Xc[q] = czero<T>();
    cta_bar();
    vcycle<T, NF, L + 1>(c, dsm);
    PINT_MGP_DISPATCH(prolong_type, c, X, Xc)
    cta_bar();
    sweeps<T, NF, L>(c, X, B, c.post, false);
  }
}

// CTAs of up to 512 threads, one per SM: 128 registers a thread (measured
// at 64 x 64 elements: 2.52 ms per 516-field launch at 512 threads against
// 2.83 ms for a 1024-thread variant with 64 registers)
template <class T, int NF>
__global__ void __launch_bounds__(512, 1) mg_q2p_kernel(MGLaunch<T> L) {
  constexpr int NL = ilog2c(NF);
  using V0 = PLev<NF, 0>;
  constexpr int n0 = 2 * NF + 1;
  __shared__ T s_w[NL * 4 * 25];
  __shared__ T s_di[NL * 4];
  __shared__ cpx<T> s_tw[100];
  __shared__ cpx<T> s_td[9];
  extern __shared__ __align__(16) unsigned char mgp_dsm[];
  const FieldJob jb = L.jobs[blockIdx.x];
  if (L.active && !L.active[jb.freq]) return;
  const OpCoef oc = L.ops[jb.op];
  // stencil weights of every level (FP64 -> T), real operator
  for (int l = 0; l < NL; ++l) {
    level_weights<T, 2>(L.t64, l, 2 * (NF >> l) + 1, mkc<double>(oc.ar, oc.ai), oc.b, s_tw, s_td);
    __syncthreads();
    for (int q = threadIdx.x; q < 100; q += blockDim.x) s_w[l * 100 + q] = s_tw[q].x;
    if (threadIdx.x < 4) s_di[l * 4 + threadIdx.x] = s_td[threadIdx.x].x;
    __syncthreads();
  }
  Ctx<T, NF> c;
  cpx<T>* ws = L.ws + (size_t)blockIdx.x * L.fields_per_job * L.lay.per_job;
  for (int l = 0; l < NL; ++l) {
    c.X[l] = ws + L.lay.off_x[l];
    c.B[l] = ws + L.lay.off_b[l];
    c.R[l] = l + 1 < NL ? ws + L.lay.off_r[l] : nullptr;
  }
  c.sw = s_w;
  c.sdi = s_di;
  c.omega = T(L.omega);
  c.pre = L.pre;
  c.post = L.post;
  type_group(c.g, c.t, c.nt);
  c.inv = L.coarse_inv + (size_t)jb.op * PINT_NC_MAX * PINT_NC_MAX * 2;
  // right-hand side into its class layout (0 off the unknowns and in padding
  // slots); zero iterate
  {
    cpx<T>* X0 = xlev<T, NF, 0>(c, mgp_dsm);
    cpx<T>* B0 = c.B[0];
    const cpx<T>* in = L.bbase + jb.b_off[0];
    for (int q = threadIdx.x; q < V0::SIZEX; q += blockDim.x) X0[q] = czero<T>();
    for (int q = threadIdx.x; q < 36 * V0::CS; q += blockDim.x) {
      const int cls = q / V0::CS, kk = q - cls * V0::CS;
      const int ty = cls / 9, rr = cls % 9;
      const int a = rr % 3 + 3 * (kk % V0::W3), b = rr / 3 + 3 * (kk / V0::W3);
      const int ix = 2 * a + (ty & 1), iy = 2 * b + (ty >> 1);
      cpx<T> v = czero<T>();
      if (ix >= 1 && iy >= 1 && ix <= n0 - 2 && iy <= n0 - 2) v = in[(size_t)iy * n0 + ix];
      B0[q] = v;
    }
  }
  __syncthreads();
  for (int cyc = 0; cyc < L.cycles; ++cyc) vcycle<T, NF, 0>(c, mgp_dsm);
  // result back to the natural layout (0 off the unknowns)
  {
    const cpx<T>* X0 = xlev<T, NF, 0>(c, mgp_dsm);
    cpx<T>* out = L.xbase + jb.x_off[0];
    for (int i = threadIdx.x; i < n0 * n0; i += blockDim.x) {
      const int ix = i % n0, iy = i / n0;
      const bool unk = ix >= 1 && iy >= 1 && ix <= n0 - 2 && iy <= n0 - 2;
      out[i] = unk ? X0[((ix & 1) + 2 * (iy & 1)) * V0::SUBX + (iy >> 1) * V0::PX + (ix >> 1)] : czero<T>();
    }
  }
}

template <class T, int NF>
bool launch_nf(const MGLaunch<T>& L, int threads, cudaStream_t st) {
  using PL = PPlan<T, NF>;
  static const bool ok = [] {
    const cudaError_t e = cudaFuncSetAttribute(mg_q2p_kernel<T, NF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)PL::BYTES);
    if (e != cudaSuccess) cudaGetLastError();
    return e == cudaSuccess;
  }();
  if (!ok) return false;
  mg_q2p_kernel<T, NF><<<L.njobs, threads > 512 ? 512 : threads, (size_t)PL::BYTES, st>>>(L);
  return true;
}

}  // namespace

// Launches the compile-time-sized velocity multigrid when it covers this
// launch (real operator W_j, no convection, finest grid of 4..256 elements
// per side, one field per job, 128..1024 threads in multiples of 128, more
// than 512 run as 512); returns false (nothing launched) otherwise.
template <class T>
bool launch_mg_q2p(const MGLaunch<T>& L, int threads, cudaStream_t st) {
  if (L.space != 2 || L.conv || L.cw || L.fields_per_job != 1 || threads < 128 || threads % 128 || threads > 1024)
    return false;
  const int N = (L.lay.n[0] - 1) / 2;
  if (L.lay.nlev != ilog2c(N) || (1 << L.lay.nlev) != N) return false;
  switch (N) {
    case 4: return launch_nf<T, 4>(L, threads, st);
    case 8: return launch_nf<T, 8>(L, threads, st);
    case 16: return launch_nf<T, 16>(L, threads, st);
    case 32: return launch_nf<T, 32>(L, threads, st);
    case 64: return launch_nf<T, 64>(L, threads, st);
    case 128: return launch_nf<T, 128>(L, threads, st);
    case 256: return launch_nf<T, 256>(L, threads, st);
    default: return false;
  }
}

// FP32 here, FP64 in k_mgp64.cu (a translation unit of its own, so that the
// build compiles the two in parallel)
#ifndef PINT_MGP_FP64
template bool launch_mg_q2p<float>(const MGLaunch<float>&, int, cudaStream_t);
#else
template bool launch_mg_q2p<double>(const MGLaunch<double>&, int, cudaStream_t);
#endif

}  // namespace pint
