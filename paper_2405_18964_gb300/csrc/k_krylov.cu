// k_krylov.cu -- Krylov machinery.
//  * Inner GMRES (Sec. 3.4, Algorithm 2): right-preconditioned complex
//    GMRES for all frequencies at once, modified Gram-Schmidt, complex
//    Givens rotations, per-frequency stopping |g_{i+1}| <= eps ||s_j||.
//    Hessenberg, rotations and the least-squares solve are FP64 on the
//    device; dot products accumulate in FP64 with a fixed reduction order.
//  * Outer FGMRES (Sec. 3.4): FP64 multi-dot / multi-axpy for classical
//    Gram-Schmidt with reorthogonalisation.
#include "krylov.h"

namespace pint {

namespace {

constexpr int RT = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum; result valid in thread 0
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
    r = warp_sum(r);
  }
  return r;
}

template <class T>
__global__ void __launch_bounds__(RT) bdot_partial(int J, long long n, const cpx<T>* A, const cpx<T>* B,
                                                   long long astride, long long bstride, double* partial,
                                                   const int* active) {
  __shared__ double sh[32];
  const int j = blockIdx.y, ch = blockIdx.x;
  if (active && !active[j]) return;
  const long long per = (n + GM_CH - 1) / GM_CH;
  const long long lo = ch * per, hi = min(n, lo + per);
  const cpx<T>* a = A + (size_t)j * astride;
  const cpx<T>* b = B + (size_t)j * bstride;
  double re = 0, im = 0;
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const cpx<T> u = a[i], v = b[i];
    // conj(u) * v
    re += (double)u.x * (double)v.x + (double)u.y * (double)v.y;
    im += (double)u.x * (double)v.y - (double)u.y * (double)v.x;
  }
  re = block_sum(re, sh);
  im = block_sum(im, sh);
  if (threadIdx.x == 0) {
    partial[((size_t)j * GM_CH + ch) * 2] = re;
    partial[((size_t)j * GM_CH + ch) * 2 + 1] = im;
  }
}

__global__ void bdot_reduce(int J, const double* partial, double* dest, long long dstride, const int* active,
                            bool norm) {
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (j >= J) return;
  if (active && !active[j]) return;
  double re = 0, im = 0;
  for (int c = lane; c < GM_CH; c += 32) {
    re += partial[((size_t)j * GM_CH + c) * 2];
    im += partial[((size_t)j * GM_CH + c) * 2 + 1];
  }
  re = warp_sum(re);
  im = warp_sum(im);
  if (lane == 0) {
    dest[(size_t)j * dstride] = norm ? sqrt(re > 0.0 ? re : 0.0) : re;
    dest[(size_t)j * dstride + 1] = norm ? 0.0 : im;
  }
}

template <class T>
__global__ void baxpy_dev_kernel(int J, long long n, const cpx<T>* A, cpx<T>* B, long long stride, const double* coef,
                                 long long cstride, double sign, const int* active) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= n) return;
  if (active && !active[j]) return;
  const cpx<T> c = mkc<T>(T(sign * coef[(size_t)j * cstride]), T(sign * coef[(size_t)j * cstride + 1]));
  const size_t q = (size_t)j * stride + i;
  B[q] = B[q] - c * A[q];
}

template <class T>
__global__ void bscale_inv_kernel(int J, long long n, const cpx<T>* W, cpx<T>* V, long long stride, const double* nrm,
                                  long long nstride, const int* active) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= n) return;
  if (active && !active[j]) return;
  const double h = nrm[(size_t)j * nstride];
  const size_t q = (size_t)j * stride + i;
  V[q] = h != 0.0 ? T(1.0 / h) * W[q] : czero<T>();
}

__global__ void gmres_start_kernel(GmresState S) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= S.J) return;
  // beta0 was written as the complex dot <s, s> at beta0-scratch (g[j][0])
  const double b2 = S.g[(size_t)j * (S.m + 1) * 2];
  const double b = sqrt(b2 > 0 ? b2 : 0.0);
  S.beta0[j] = b;
  for (int i = 0; i <= S.m; ++i) {
    S.g[((size_t)j * (S.m + 1) + i) * 2] = (i == 0) ? b : 0.0;
    S.g[((size_t)j * (S.m + 1) + i) * 2 + 1] = 0.0;
  }
  S.active[j] = b > 0.0 ? 1 : 0;
  S.its[j] = 0;
}

__global__ void gmres_givens_kernel(GmresState S, int i, double tol, int fixed) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= S.J) return;
  if (!S.active[j]) return;
  const int m = S.m;
  double* Hc = S.H + (size_t)j * (m + 1) * m * 2;  // column i entries at row r: (r*m + i)*2
  auto Hr = [&](int r) -> double* { return Hc + ((size_t)r * m + i) * 2; };
  double* cs = S.cs + (size_t)j * m;
  double* sn = S.sn + (size_t)j * m * 2;
  double* g = S.g + (size_t)j * (m + 1) * 2;
  const double hn = Hr(i + 1)[0];
  for (int l = 0; l < i; ++l) {
    double* h0 = Hr(l);
    double* h1 = Hr(l + 1);
    const double c = cs[l], sr = sn[2 * l], si = sn[2 * l + 1];
    // t = c h0 + s h1 ; h1' = -conj(s) h0 + c h1
    const double tr = c * h0[0] + (sr * h1[0] - si * h1[1]);
    const double ti = c * h0[1] + (sr * h1[1] + si * h1[0]);
    const double ur = -(sr * h0[0] + si * h0[1]) + c * h1[0];
    const double ui = -(sr * h0[1] - si * h0[0]) + c * h1[1];
    h0[0] = tr;
    h0[1] = ti;
    h1[0] = ur;
    h1[1] = ui;
  }
  double* a = Hr(i);
  double* b = Hr(i + 1);
  const double ar = a[0], ai = a[1], br = b[0], bi = b[1];
  const double aa = sqrt(ar * ar + ai * ai), ab = sqrt(br * br + bi * bi);
  double c, sr, si, rr, ri;
  if (ab == 0.0) {
    c = 1.0;
    sr = si = 0.0;
    rr = ar;
    ri = ai;
  } else if (aa == 0.0) {
    c = 0.0;
    sr = br / ab;
    si = -bi / ab;
    rr = ab;
    ri = 0.0;
  } else {
    const double t = sqrt(aa * aa + ab * ab);
    const double pr = ar / aa, pi = ai / aa;  // phase of a
    c = aa / t;
    // s = ph * conj(b) / t
    sr = (pr * br + pi * bi) / t;
    si = (pi * br - pr * bi) / t;
    rr = pr * t;
    ri = pi * t;
  }
  cs[i] = c;
  sn[2 * i] = sr;
  sn[2 * i + 1] = si;
  a[0] = rr;
  a[1] = ri;
  b[0] = 0.0;
  b[1] = 0.0;
  // g_{i+1} = -conj(s) g_i ; g_i = c g_i
  const double gr = g[2 * i], gi = g[2 * i + 1];
  g[2 * (i + 1)] = -(sr * gr + si * gi);
  g[2 * (i + 1) + 1] = -(sr * gi - si * gr);
  g[2 * i] = c * gr;
  g[2 * i + 1] = c * gi;
  S.its[j] = i + 1;
  const double res = sqrt(g[2 * (i + 1)] * g[2 * (i + 1)] + g[2 * (i + 1) + 1] * g[2 * (i + 1) + 1]);
  bool done = fixed > 0 ? (i + 1 >= fixed) : (res <= tol * S.beta0[j]);
  if (hn == 0.0 || i + 1 >= m) done = true;
  if (done)
    S.active[j] = 0;
  else
    atomicAdd(S.count, 1);
}

__global__ void gmres_solve_kernel(GmresState S) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= S.J) return;
  const int m = S.m, k = S.its[j];
  const double* H = S.H + (size_t)j * (m + 1) * m * 2;
  const double* g = S.g + (size_t)j * (m + 1) * 2;
  double* y = S.y + (size_t)j * m * 2;
  for (int l = k - 1; l >= 0; --l) {
    double sr = g[2 * l], si = g[2 * l + 1];
    for (int q = l + 1; q < k; ++q) {
      const double hr = H[((size_t)l * m + q) * 2], hi = H[((size_t)l * m + q) * 2 + 1];
      sr -= hr * y[2 * q] - hi * y[2 * q + 1];
      si -= hr * y[2 * q + 1] + hi * y[2 * q];
    }
    const double dr = H[((size_t)l * m + l) * 2], di = H[((size_t)l * m + l) * 2 + 1];
    const double den = dr * dr + di * di;
    y[2 * l] = (sr * dr + si * di) / den;
    y[2 * l + 1] = (si * dr - sr * di) / den;
  }
}

template <class T>
__global__ void gmres_combine_kernel(GmresState S, long long n, const cpx<T>* Z, long long zstride_l, cpx<T>* x) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= n) return;
  const int k = S.its[j];
  const double* y = S.y + (size_t)j * S.m * 2;
  double re = 0, im = 0;
  for (int l = 0; l < k; ++l) {
    const cpx<T> z = Z[(size_t)l * zstride_l + (size_t)j * n + i];
    re += y[2 * l] * (double)z.x - y[2 * l + 1] * (double)z.y;
    im += y[2 * l] * (double)z.y + y[2 * l + 1] * (double)z.x;
  }
  x[(size_t)j * n + i] = mkc<T>(T(re), T(im));
}

// ---- classical Gram-Schmidt over the batched basis ---------------------------
constexpr int GB = 8;  // basis vectors per pass of the dot kernel

template <class T>
__global__ void __launch_bounds__(RT) bmdot_partial(int J, long long n, const cpx<T>* V, long long vstride, int l0,
                                                    int cnt, const cpx<T>* w, double* partial, const int* active) {
  __shared__ double sh[32];
  const int j = blockIdx.y, ch = blockIdx.x;
  if (active && !active[j]) return;
  const long long per = (n + GM_CH - 1) / GM_CH;
  const long long lo = ch * per, hi = min(n, lo + per);
  const cpx<T>* wj = w + (size_t)j * n;
  // per-thread partial sums in T over a few elements, reduced in FP64
  T re[GB], im[GB];
#pragma unroll
  for (int q = 0; q < GB; ++q) re[q] = im[q] = T(0);
  for (long long e = lo + threadIdx.x; e < hi; e += blockDim.x) {
    const cpx<T> v = wj[e];
#pragma unroll
    for (int q = 0; q < GB; ++q)
      if (l0 + q < cnt) {
        const cpx<T> u = V[(size_t)(l0 + q) * vstride + (size_t)j * n + e];
        re[q] = fma(u.x, v.x, fma(u.y, v.y, re[q]));  // conj(u) v
        im[q] = fma(u.x, v.y, fma(-u.y, v.x, im[q]));
      }
  }
  for (int q = 0; q < GB && l0 + q < cnt; ++q) {
    const double a = block_sum((double)re[q], sh);
    const double b = block_sum((double)im[q], sh);
    if (threadIdx.x == 0) {
      double* p = partial + (((size_t)j * GM_CH + ch) * cnt + (l0 + q)) * 2;
      p[0] = a;
      p[1] = b;
    }
  }
}

__global__ void bmdot_reduce(int J, int cnt, const double* partial, double* H, long long hs, int m, int col,
                             bool add, const int* active) {
  const int j = blockIdx.y;
  const int l = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (l >= cnt) return;
  if (active && !active[j]) return;
  double re = 0, im = 0;
  for (int c = lane; c < GM_CH; c += 32) {
    re += partial[(((size_t)j * GM_CH + c) * cnt + l) * 2];
    im += partial[(((size_t)j * GM_CH + c) * cnt + l) * 2 + 1];
  }
  re = warp_sum(re);
  im = warp_sum(im);
  if (lane == 0) {
    double* h = H + (size_t)j * hs + ((size_t)l * m + col) * 2;
    if (add) {
      h[0] += re;
      h[1] += im;
    } else {
      h[0] = re;
      h[1] = im;
    }
  }
}

// coefficients of the current pass are the last written ones: for the first
// pass H itself, for the second pass the increment is passed separately
template <class T>
__global__ void __launch_bounds__(RT) bmaxpy_kernel(int J, long long n, const cpx<T>* V, long long vstride,
                                                    int cnt, cpx<T>* w, const double* coef, long long cs_j,
                                                    double* nrm_partial, const int* active) {
  __shared__ double sh[32];
  __shared__ cpx<T> hc[128];
  const int j = blockIdx.y, ch = blockIdx.x;
  if (active && !active[j]) return;
  for (int l = threadIdx.x; l < cnt; l += blockDim.x)
    hc[l] = mkc<T>(T(coef[(size_t)j * cs_j + 2 * l]), T(coef[(size_t)j * cs_j + 2 * l + 1]));
  __syncthreads();
  const long long per = (n + GM_CH - 1) / GM_CH;
  const long long lo = ch * per, hi = min(n, lo + per);
  cpx<T>* wj = w + (size_t)j * n;
  T nr = T(0);
  for (long long e = lo + threadIdx.x; e < hi; e += blockDim.x) {
    cpx<T> acc = wj[e];
    for (int l = 0; l < cnt; ++l) acc = acc - hc[l] * V[(size_t)l * vstride + (size_t)j * n + e];
    wj[e] = acc;
    nr = fma(acc.x, acc.x, fma(acc.y, acc.y, nr));
  }
  if (nrm_partial) {
    const double t = block_sum((double)nr, sh);
    if (threadIdx.x == 0) nrm_partial[(size_t)j * GM_CH + ch] = t;
  }
}

// copy one H column (rows 0..cnt-1) into a contiguous coefficient buffer
__global__ void hcol_gather(int J, int cnt, const double* H, long long hs, int m, int col, double* out,
                            const int* active) {
  const int j = blockIdx.x;
  if (active && !active[j]) return;
  for (int l = threadIdx.x; l < cnt; l += blockDim.x) {
    out[((size_t)j * 128 + l) * 2] = H[(size_t)j * hs + ((size_t)l * m + col) * 2];
    out[((size_t)j * 128 + l) * 2 + 1] = H[(size_t)j * hs + ((size_t)l * m + col) * 2 + 1];
  }
}

__global__ void hcol_add(int J, int cnt, double* H, long long hs, int m, int col, const double* inc,
                         const int* active) {
  const int j = blockIdx.x;
  if (active && !active[j]) return;
  for (int l = threadIdx.x; l < cnt; l += blockDim.x) {
    H[(size_t)j * hs + ((size_t)l * m + col) * 2] += inc[((size_t)j * 128 + l) * 2];
    H[(size_t)j * hs + ((size_t)l * m + col) * 2 + 1] += inc[((size_t)j * 128 + l) * 2 + 1];
  }
}

__global__ void nrm_reduce(int J, const double* nrm_partial, double* nrm, long long ns, const int* active) {
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (j >= J) return;
  if (active && !active[j]) return;
  double s = 0;
  for (int c = lane; c < GM_CH; c += 32) s += nrm_partial[(size_t)j * GM_CH + c];
  s = warp_sum(s);
  if (lane == 0) {
    nrm[(size_t)j * ns] = sqrt(s > 0.0 ? s : 0.0);
    nrm[(size_t)j * ns + 1] = 0.0;
  }
}

// ---- outer ------------------------------------------------------------------
constexpr int MB = 8;  // vectors per multi-dot pass

__global__ void __launch_bounds__(RT) mdot_partial(const double* V, int cnt, const double* w, long long n,
                                                   double* partial) {
  __shared__ double sh[32];
  const long long per = (n + gridDim.x - 1) / gridDim.x;
  const long long lo = blockIdx.x * per, hi = min(n, lo + per);
  double acc[MB];
#pragma unroll
  for (int l = 0; l < MB; ++l) acc[l] = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const double wi = w[i];
#pragma unroll
    for (int l = 0; l < MB; ++l)
      if (l < cnt) acc[l] = fma(V[(size_t)l * n + i], wi, acc[l]);
  }
  for (int l = 0; l < cnt; ++l) {
    const double s = block_sum(acc[l], sh);
    if (threadIdx.x == 0) partial[(size_t)l * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void mdot_reduce(const double* partial, int nparts, double* h) {
  __shared__ double sh[32];
  const int l = blockIdx.x;
  double s = 0.0;
  for (int c = threadIdx.x; c < nparts; c += blockDim.x) s += partial[(size_t)l * nparts + c];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) h[l] = s;
}

__global__ void maxpy_kernel(const double* V, int cnt, const double* h, double* w, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = w[i];
  for (int l = 0; l < cnt; ++l) s = fma(-h[l], V[(size_t)l * n + i], s);
  w[i] = s;
}

__global__ void axpby_kernel(double a, const double* x, double b, double* y, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = a * x[i] + b * y[i];
}

__global__ void scale_inv_dev_kernel(const double* x, const double* s, double* y, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const double v = s[0];
    y[i] = v != 0.0 ? x[i] / v : 0.0;
  }
}

inline unsigned nb(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

template <class T>
void launch_bdot(int J, long long n, const cpx<T>* A, const cpx<T>* B, long long astride, long long bstride,
                 double* partial, double* dest, long long dstride, const int* active, bool norm,
                 cudaStream_t st) {
  bdot_partial<T><<<dim3(GM_CH, J), RT, 0, st>>>(J, n, A, B, astride, bstride, partial, active);
  bdot_reduce<<<nb(J, 8), 256, 0, st>>>(J, partial, dest, dstride, active, norm);
}

template <class T>
void launch_baxpy_dev(int J, long long n, const cpx<T>* A, cpx<T>* B, long long stride, const double* coef,
                      long long cstride, double sign, const int* active, cudaStream_t st) {
  baxpy_dev_kernel<T><<<dim3(nb(n, RT), J), RT, 0, st>>>(J, n, A, B, stride, coef, cstride, sign, active);
}

template <class T>
void launch_bscale_inv(int J, long long n, const cpx<T>* W, cpx<T>* V, long long stride, const double* nrm,
                       long long nstride, const int* active, cudaStream_t st) {
  bscale_inv_kernel<T><<<dim3(nb(n, RT), J), RT, 0, st>>>(J, n, W, V, stride, nrm, nstride, active);
}

void launch_gmres_start(GmresState& S, cudaStream_t st) { gmres_start_kernel<<<nb(S.J, 128), 128, 0, st>>>(S); }

void launch_gmres_givens(GmresState& S, int i, double tol, int fixed, cudaStream_t st) {
  cudaMemsetAsync(S.count, 0, sizeof(int), st);
  gmres_givens_kernel<<<nb(S.J, 128), 128, 0, st>>>(S, i, tol, fixed);
}

template <class T>
void launch_gmres_finish(GmresState& S, long long n, const cpx<T>* Z, long long zstride_l, cpx<T>* x,
                         cudaStream_t st) {
  gmres_solve_kernel<<<nb(S.J, 128), 128, 0, st>>>(S);
  gmres_combine_kernel<T><<<dim3(nb(n, RT), S.J), RT, 0, st>>>(S, n, Z, zstride_l, x);
}

template <class T>
void launch_bmdot(int J, long long n, const cpx<T>* V, long long vstride, int cnt, const cpx<T>* w,
                  double* partial, double* H, long long hs, int m, int col, bool add, const int* active,
                  cudaStream_t st) {
  for (int l0 = 0; l0 < cnt; l0 += GB)
    bmdot_partial<T><<<dim3(GM_CH, J), RT, 0, st>>>(J, n, V, vstride, l0, cnt, w, partial, active);
  bmdot_reduce<<<dim3((cnt + 7) / 8, J), 256, 0, st>>>(J, cnt, partial, H, hs, m, col, add, active);
}

template <class T>
void launch_bmaxpy(int J, long long n, const cpx<T>* V, long long vstride, int cnt, cpx<T>* w,
                   const double* coef, long long cs_j, double* nrm_partial, double* nrm, long long ns,
                   const int* active, cudaStream_t st) {
  bmaxpy_kernel<T><<<dim3(GM_CH, J), RT, 0, st>>>(J, n, V, vstride, cnt, w, coef, cs_j, nrm_partial, active);
  if (nrm_partial) nrm_reduce<<<nb(J, 8), 256, 0, st>>>(J, nrm_partial, nrm, ns, active);
}

void launch_hcol_gather(int J, int cnt, const double* H, long long hs, int m, int col, double* out,
                        const int* active, cudaStream_t st) {
  hcol_gather<<<J, 128, 0, st>>>(J, cnt, H, hs, m, col, out, active);
}

void launch_hcol_add(int J, int cnt, double* H, long long hs, int m, int col, const double* inc,
                     const int* active, cudaStream_t st) {
  hcol_add<<<J, 128, 0, st>>>(J, cnt, H, hs, m, col, inc, active);
}

void launch_mdot(const double* V, int cnt, const double* w, long long n, double* partial, double* h,
                 cudaStream_t st) {
  for (int l0 = 0; l0 < cnt; l0 += MB) {
    const int c = cnt - l0 < MB ? cnt - l0 : MB;
    mdot_partial<<<MDOT_CTAS, RT, 0, st>>>(V + (size_t)l0 * n, c, w, n, partial);
    mdot_reduce<<<c, RT, 0, st>>>(partial, MDOT_CTAS, h + l0);
  }
}

void launch_maxpy(const double* V, int cnt, const double* h, double* w, long long n, cudaStream_t st) {
  maxpy_kernel<<<nb(n, RT), RT, 0, st>>>(V, cnt, h, w, n);
}

void launch_axpby(double a, const double* x, double b, double* y, long long n, cudaStream_t st) {
  axpby_kernel<<<nb(n, RT), RT, 0, st>>>(a, x, b, y, n);
}

void launch_scale_inv_dev(const double* x, const double* s, double* y, long long n, cudaStream_t st) {
  scale_inv_dev_kernel<<<nb(n, RT), RT, 0, st>>>(x, s, y, n);
}

#define PINT_INST(T)                                                                                         \
  template void launch_bdot<T>(int, long long, const cpx<T>*, const cpx<T>*, long long, long long, double*, \
                               double*, long long, const int*, bool, cudaStream_t);                         \
  template void launch_baxpy_dev<T>(int, long long, const cpx<T>*, cpx<T>*, long long, const double*,       \
                                    long long, double, const int*, cudaStream_t);                           \
  template void launch_bscale_inv<T>(int, long long, const cpx<T>*, cpx<T>*, long long, const double*,      \
                                     long long, const int*, cudaStream_t);                                  \
  template void launch_gmres_finish<T>(GmresState&, long long, const cpx<T>*, long long, cpx<T>*,           \
                                       cudaStream_t);                                                       \
  template void launch_bmdot<T>(int, long long, const cpx<T>*, long long, int, const cpx<T>*, double*,      \
                                double*, long long, int, int, bool, const int*, cudaStream_t);               \
  template void launch_bmaxpy<T>(int, long long, const cpx<T>*, long long, int, cpx<T>*, const double*,     \
                                 long long, double*, double*, long long, const int*, cudaStream_t);
PINT_INST(float)
PINT_INST(double)
#undef PINT_INST

}  // namespace pint
