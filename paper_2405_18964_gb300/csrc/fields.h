// fields.h -- launchers for field-wise kernels (internal).
#pragma once
#include "common.cuh"

namespace pint {

// Slot offsets (elements) of the six fields inside one block of n_blk.
struct Slots {
  long long vx, vy, p, lx, ly, mu, nblk;
  int ns, nq, n2, n1;
};

// ---- FP64 time-domain KKT matvec (Eq. FinalA) --------------------------
struct KKTArgs {
  Tabs<double> tabs;
  Slots s;
  int K;
  double tau, beta, nu;
  bool conv;           // separable recirculating wind
  const double* nst;   // or node-order FP64 convection stencils [ns][25] (general wind), else null
  const double* x;
  double* y;
};
void launch_kkt_matvec(const KKTArgs& a, cudaStream_t st);

// ---- per-frequency block matvec (Eq. SubBlockG, or Z_j of the Stokes
// transform), complex, precision T.  Per-frequency coefficients:
//   row1 = a11 M v + a12 M lam + g12 (nu K lam - N lam) + dl B^T mu
//   row2 = a21 M v + g21 (nu K v + N v) + a22 M lam + dl B^T p
//   row3 = dl B lam ; row4 = dl B v
struct BlkCoef {
  double a11r, a11i, a12r, a12i, a21r, a21i, a22r, a22i, g12, g21, dl, pad;
};
template <class T>
struct BlkArgs {
  Tabs<T> tabs;
  const T* n2d;  // per-node Q2 convection rows [blocked node][25] (conv only)
  Slots s;
  int J;
  double nu;
  bool conv;
  const BlkCoef* coef;
  const int* active;
  const cpx<T>* x;
  cpx<T>* y;
};
template <class T>
void launch_block_matvec(const BlkArgs<T>& a, cudaStream_t st);

// ---- operator combinations on frequency fields -------------------------
// Each row: out[out_slot] = w * z[z_slot] + sum_t (a_t M + b_t K + c_t N) x[in_slot_t]
// coefficient index zc / tc[t] into the table coef[J][ncoef] (w = coef.ar + i coef.ai).
struct ComboRow {
  long long out_slot, z_slot, in_slot[2];
  int zc, tc[2], nt, has_z;
};
template <class T>
struct ComboArgs {
  Tabs<T> tabs;
  const T* n2d;   // per-node Q2 convection rows [blocked node][25] (conv only)
  const T* np2d;  // per-node Q1 convection rows [node][9] (conv only)
  Slots s;
  int J, nrows, ncoef, space;  // space: 2 = Q2 field rows, 1 = Q1 field rows
  bool conv;
  ComboRow rows[4];
  const OpCoef* coef;
  const int* active;
  const cpx<T>* x;
  const cpx<T>* z;
  cpx<T>* out;
};
template <class T>
void launch_combo(const ComboArgs<T>& a, cudaStream_t st);

// out[p_slot] = z[zp] + c * B(x[velA]) ; out[mu_slot] = z[zmu] + c * B(x[velB])
// (velA / velB: slot of the x component; the y component follows at +ns)
template <class T>
struct BResArgs {
  Tabs<T> tabs;
  Slots s;
  int J;
  double c;
  const double* cj;  // per-frequency c (replaces c when set)
  long long out0, z0, vel0, out1, z1, vel1;
  const int* active;
  const cpx<T>* x;
  const cpx<T>* z;
  cpx<T>* out;
};
template <class T>
void launch_bres(const BResArgs<T>& a, cudaStream_t st);

// out[j][so + i] = al_j * A[j][sa + i] + be_j * B[j][sb + i], i < len
// (al, be: complex tables [J] of (re, im) pairs; B may be null)
template <class T>
void launch_lincomb(int J, long long nblk, long long len, cpx<T>* out, long long so, const cpx<T>* A, long long sa,
                    const double* al, const cpx<T>* B, long long sb, const double* be, const int* active,
                    cudaStream_t st);

// Stokes transforms: dir = 0 applies (T_j^l)^{-1}, dir = 1 applies (T_j^r)^{-1}
// in place.  tc: per-frequency (sqrt(tau), d_c, c_2) triples.
template <class T>
void launch_stokes_transform(int dir, int J, const Slots& s, const double* tc, cpx<T>* x, cudaStream_t st);

// ---- time DFT along the block index ------------------------------------
template <class T>
void launch_dft_forward(int K, int J, long long nblk, const double* x, cpx<T>* X, const T* cosk, const T* sink,
                        cudaStream_t st);
template <class T>
void launch_dft_inverse(int K, int J, long long nblk, const cpx<T>* X, double* y, const T* cosk, const T* sink,
                        cudaStream_t st);

// ---- right-hand side (Sec. 2.2 backward-Euler equations) ----------------
// b: adjoint rows tau M v_d(t_k); state rows tau M f(t_k), first state row
// also M v_0.  vd, f: [K][2][ns]; v0: [2][ns]; only interior nodal values
// enter (the data are vectors of the velocity unknowns).  f, v0 may be null.
struct RhsArgs {
  Tabs<double> tabs;
  Slots s;
  int K;
  double tau;
  const double* vd;
  const double* f;
  const double* v0;
  double* b;
  int full;  // 1: loads use every nodal value (M_{I,:}); 0: boundary values dropped
};
void launch_rhs(const RhsArgs& a, cudaStream_t st);
// x (K blocks, zeroed by the caller) gets the boundary nodal values of
// g [K][2][ns] in its state-velocity slots; interior entries stay 0.
void launch_lift_scatter(const Slots& s, int K, const double* g, double* x, cudaStream_t st);

// ---- misc ----------------------------------------------------------------
// Zero the non-unknown entries (Dirichlet velocity nodes, pinned pressure)
// of nvec consecutive blocks; real (ncomp = 1) or complex (ncomp = 2) data.
void launch_mask_blocks(const Slots& s, long long nvec, int ncomp, double* x, cudaStream_t st);
void launch_copy_d2f(const double* a, float* b, long long n, cudaStream_t st);
void launch_copy_f2d(const float* a, double* b, long long n, cudaStream_t st);
// count of non-finite entries (atomic) of a double array
void launch_count_nonfinite(const double* a, long long n, int* count, cudaStream_t st);

}  // namespace pint
