// kernels.h -- host-side launchers of the device kernels (internal).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace pint {

// One multigrid / Chebyshev job: a scalar field of one frequency.
// Offsets are in complex elements, relative to the base pointers of the launch.
struct FieldJob {
  long long x_off;
  long long b_off;
  int op;
  int freq;
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
};

#define PINT_NC_MAX 9

template <class T>
void launch_mg(const MGLaunch<T>& L, cudaStream_t st);

template <class T>
struct ChebLaunch {
  Tabs<T> tabs;
  const FieldJob* jobs;
  int njobs;
  cpx<T>* xbase;
  const cpx<T>* bbase;
  cpx<T>* ws;         // 2 fields per job
  long long per_job;  // complex elements per job
  const int* active;
  int steps;
  double lmin, lmax;
  int space;
};

template <class T>
void launch_cheb(const ChebLaunch<T>& L, cudaStream_t st);

// Coarse-grid inverses: for each op, the dense inverse of the operator on
// the coarsest grid (FP64, Gauss-Jordan with partial pivoting).
void launch_coarse_setup(const Tabs<double>& tabs, const OpCoef* ops, const int* op_space,
                         const int* op_conv, int nops, double* inv, int* status, cudaStream_t st);

}  // namespace pint
