// kernels.h -- host-side launchers of the device kernels (internal).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "common.cuh"

namespace pint {

// One multigrid / Chebyshev job: up to PINT_MAXF scalar fields of one
// frequency that share one operator.  Offsets are in complex elements,
// relative to the base pointers of the launch.
#define PINT_MAXF 4
struct FieldJob {
  long long x_off[PINT_MAXF];
  long long b_off[PINT_MAXF];
  int nf;
  int op;
  int freq;
  int pad;
};

// Per-level workspace offsets (complex elements) inside one job's workspace.
struct MGLayout {
  int nlev;                        // levels, finest = 0
  int n[PINT_MAXLEV];              // nodes per side at each level
  long long off_x[PINT_MAXLEV];    // level >= 1
  long long off_b[PINT_MAXLEV];    // level >= 1
  long long off_r[PINT_MAXLEV];    // level <= nlev-2
  long long per_job;               // complex elements per job
};

template <class T>
struct MGLaunch {
  Tabs<T> tabs;
  Tabs<double> t64;          // FP64 bands: stencil weights are formed in FP64
  const T* n2d[PINT_MAXLEV]; // Q2 convection stencil per blocked node [n^2][25] (conv only)
  int fields_per_job;        // workspace slots per job
  bool cw;                   // complex operator coefficient (Oseen shifts)
  MGLayout lay;
  const OpCoef* ops;
  const double* coarse_inv;  // complex FP64, [op][PINT_NC_MAX^2][2]
  const FieldJob* jobs;
  int njobs;
  cpx<T>* xbase;
  const cpx<T>* bbase;
  cpx<T>* ws;
  const int* active;  // per-frequency flags or nullptr
  int cycles, pre, post;
  double omega;
  int space;  // 2 = Q2 (velocity component), 1 = Q1 (pressure)
  bool conv;
  int active_jobs;  // > 0: jobs whose frequency is still active (sizes the CTAs), 0: all
  bool no_tune;     // true: fixed CTA size, the autotuner is not consulted (it would allocate on first use)
  unsigned smem_levels;  // Q2 multigrid: bit l set = level l's iterate in shared memory (set by launch_mg)
};

#define PINT_NC_MAX 9

template <class T>
void launch_mg(const MGLaunch<T>& L, cudaStream_t st);
// Row pitch of one node type's iterate sub-grid in the compile-time-sized
// velocity multigrid (k_mgp.cu), for a level of N elements per side: the
// smallest P >= N + 1 with P = ceil((N + 1) / 3) (mod 16), so that the nodes
// of one colour, taken in order, fall into distinct shared-memory banks;
// N + 1 for the small levels.
__host__ __device__ constexpr int q2p_pitch(int N) {
  const int w3 = (N + 3) / 3;
  if (w3 <= 4) return N + 1;
  int p = N + 1;
  while (p % 16 != w3 % 16) ++p;
  return p;
}

// The compile-time-sized velocity multigrid (k_mgp.cu) for the launches it
// covers; false (nothing launched) for the others.
template <class T>
bool launch_mg_q2p(const MGLaunch<T>& L, int threads, cudaStream_t st);
// The compile-time-sized pressure multigrid (k_mgq1.cu) for the launches it
// covers; false (nothing launched) for the others.
template <class T>
bool launch_mg_q1p(const MGLaunch<T>& L, int threads, cudaStream_t st);
// CTA-size autotuner of launch_mg (on by default) and its decisions as text.
void mg_autotune_enable(bool on);
// Fixed launch choice while the tuner is off (threads 0 = by job count;
// staging -1 = whenever possible, 0 = never, 1 = whenever possible).
void mg_fixed_config(int threads, int staging);
std::string mg_autotune_report();

template <class T>
struct ChebLaunch {
  Tabs<T> tabs;
  Tabs<double> t64;
  const FieldJob* jobs;
  int njobs;
  cpx<T>* xbase;
  const cpx<T>* bbase;
  cpx<T>* ws;         // 2 fields (r, d) per job field
  long long per_job;  // complex elements per job field
  int fields_per_job;
  const int* active;
  int steps;
  double lmin, lmax;
  int space;
  int active_jobs;  // > 0: jobs whose frequency is still active (sizes the CTAs), 0: all
};

template <class T>
void launch_cheb(const ChebLaunch<T>& L, cudaStream_t st);

// Per-node Q2 convection stencil, formed in FP64 and rounded once:
// out[b(ix, iy) * 25 + dy * 5 + dx] at level l, with b the class-blocked node
// index of the multigrid layout.  src == nullptr: the recirculating wind's
// separable N = 2 (W1 (x) X1 - X1 (x) W1); else src holds the FP64 stencils
// of this level in node order, src[(iy * n2 + ix) * 25 + dy * 5 + dx].
template <class T>
void launch_build_n2d(const Tabs<double>& t64, int l, T* out, const double* src, cudaStream_t st);

// Per-node Q1 convection stencil on the finest pressure grid, FP64 -> T:
// out[(iy * n1 + ix) * 9 + dy * 3 + dx]; from the separable
// N_p = 2 (W1 (x) X1 - X1 (x) W1) when src == nullptr, else copied from src
// (same order).
template <class T>
void launch_build_np2d(const Tabs<double>& t64, T* out, const double* src, cudaStream_t st);

// Coarse-grid inverses: for each op, the dense inverse of the operator on
// the coarsest grid (FP64, Gauss-Jordan with partial pivoting).  conv_last:
// node-order FP64 convection stencils of the coarsest Q2 grid, or nullptr for
// the separable recirculating wind.
void launch_coarse_setup(const Tabs<double>& tabs, const OpCoef* ops, const int* op_space,
                         const int* op_conv, int nops, double* inv, int* status, const double* conv_last,
                         cudaStream_t st);

}  // namespace pint
