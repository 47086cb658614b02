// krylov.h -- launchers for the Krylov kernels (internal).
#pragma once
#include "common.cuh"

namespace pint {

// Batched inner GMRES state (one system per frequency j), FP64.
struct GmresState {
  int J, m;           // frequencies, maximum iterations
  double* H;          // [J][m+1][m] complex (re, im)
  double* g;          // [J][m+1] complex
  double* cs;         // [J][m]
  double* sn;         // [J][m] complex
  double* beta0;      // [J]
  double* y;          // [J][m] complex
  double* partial;    // [J][CH] complex reduction scratch
  int* active;        // [J]
  int* its;           // [J]
  int* count;         // [1]
  double* hc;         // [J][128] complex: gathered Gram-Schmidt coefficients
  double* hc2;        // [J][128] complex: second-pass increments
  double* npart;      // [J][GM_CH] norm partial sums
  double* cpart;      // [J][GM_CH][m+1] complex dot partials
};
constexpr int GM_CH = 32;  // reduction chunks per frequency

// dest[j] = sum_i conj(A[j][i]) B[j][i] (complex FP64), written at
// dest + j * dstride (re, im); only for active j (or all if active null).
// norm = true writes (sqrt(Re dest), 0) instead (use with A == B).
template <class T>
void launch_bdot(int J, long long n, const cpx<T>* A, const cpx<T>* B, long long astride, long long bstride,
                 double* partial, double* dest, long long dstride, const int* active, bool norm,
                 cudaStream_t st);
// B[j] -= coef[j * cstride] * A[j]  (coef complex FP64 on the device)
template <class T>
void launch_baxpy_dev(int J, long long n, const cpx<T>* A, cpx<T>* B, long long stride, const double* coef,
                      long long cstride, double sign, const int* active, cudaStream_t st);
// V[j] = W[j] / nrm[j * nstride]   (nrm: the real part of a complex FP64 entry)
template <class T>
void launch_bscale_inv(int J, long long n, const cpx<T>* W, cpx<T>* V, long long stride, const double* nrm,
                       long long nstride, const int* active, cudaStream_t st);
// Start: beta0[j] = ||s_j|| (from dest), g = (beta0, 0...), active = beta0 > 0
void launch_gmres_start(GmresState& S, cudaStream_t st);
// Givens update of column i for all active j; decrements nothing, counts
// the frequencies that stay active into *count (zeroed by the launcher).
void launch_gmres_givens(GmresState& S, int i, double tol, int fixed, cudaStream_t st);
// y_j = H_j^{-1} g_j (triangular, size its[j]); x[j] = sum_l y_l Z_l[j]
template <class T>
void launch_gmres_finish(GmresState& S, long long n, const cpx<T>* Z, long long zstride_l, cpx<T>* x,
                         cudaStream_t st);

// Classical Gram-Schmidt step for all active frequencies against the basis
// V_0..V_cnt-1 (V_l = V + l * vstride, frequency j at + j * n):
//   add = false: H[j][l][col] = <V_l, w>      add = true: H[j][l][col] += <V_l, w>
// (H complex FP64 with per-frequency stride hs and row stride m).
// partial: [J][GM_CH][cnt] complex scratch.
template <class T>
void launch_bmdot(int J, long long n, const cpx<T>* V, long long vstride, int cnt, const cpx<T>* w,
                  double* partial, double* H, long long hs, int m, int col, bool add, const int* active,
                  cudaStream_t st);
// w_j -= sum_l h_{j,l} V_l (h = H column col, pass `pass` coefficients), and,
// if nrm != null, the per-chunk partial sums of |w_j|^2 after the update
// into nrm_partial[j][GM_CH]; the reduce writes sqrt into nrm[j * ns].
// coef: per-frequency contiguous complex coefficients (frequency j at
// coef + j * cs_j), at most 128 of them.
template <class T>
void launch_bmaxpy(int J, long long n, const cpx<T>* V, long long vstride, int cnt, cpx<T>* w,
                   const double* coef, long long cs_j, double* nrm_partial, double* nrm, long long ns,
                   const int* active, cudaStream_t st);
// out[j][l] = H[j][l][col] for l < cnt (complex), out stride 128 per frequency
void launch_hcol_gather(int J, int cnt, const double* H, long long hs, int m, int col, double* out,
                        const int* active, cudaStream_t st);

// H[j][l][col] += inc[j][l] (inc stride 128 per frequency)
void launch_hcol_add(int J, int cnt, double* H, long long hs, int m, int col, const double* inc,
                     const int* active, cudaStream_t st);

// ---- outer FP64 vectors --------------------------------------------------
// h[l] = <V_l, w> for l < cnt, V_l = V + l * n
void launch_mdot(const double* V, int cnt, const double* w, long long n, double* partial, double* h,
                 cudaStream_t st);
// w -= sum_l h[l] V_l
void launch_maxpy(const double* V, int cnt, const double* h, double* w, long long n, cudaStream_t st);
// y = a * x + b * y
void launch_axpby(double a, const double* x, double b, double* y, long long n, cudaStream_t st);
// y = x * (1 / s[0])  (s on device)
void launch_scale_inv_dev(const double* x, const double* s, double* y, long long n, cudaStream_t st);
constexpr int MDOT_CTAS = 1024;

}  // namespace pint
