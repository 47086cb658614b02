// dft_tc.h -- time DFT of the FP32 preconditioner on the tensor cores (internal).
//
// The circulant C = F^{-1} D F (Sec. 3.1) is diagonalised by the DFT along the
// time axis.  For real data the K complex outputs X_j, j = 0..K-1, carry K real
// degrees of freedom: Re X_j for j = 0..J-1 and Im X_j for j = 1..K-J, with
// J = floor(K/2) + 1 (Im X_0 = 0, and Im X_{K/2} = 0 for even K; the rest
// follow from X_{K-j} = conj(X_j)).  Both directions are therefore one real
// contraction with a constant matrix:
//   forward   D[i][o] = sum_k  x_k(i) F[o][k],  o < J: cos(2 pi o k / K),
//                                               o >= J: -sin(2 pi (o-J+1) k / K)
//   inverse   y_k(i)  = sum_c  a_c(i) G[k][c],  c = 2j + part of X_j(i),
//             G[k][2j] = w_j cos(2 pi j k / K) / K, G[k][2j+1] = -w_j sin(...) / K,
//             w_j = 1 for j = 0 and j = K/2, else 2.
// i runs over the n_blk spatial storage slots of one time block.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace pint {

// Operand splitting scheme (values of pint_dft_mode).
enum { DFT_TC_BF16X6 = 2, DFT_TC_TF32X3 = 3 };

struct DftTc {
  int scheme = 0;             // DFT_TC_BF16X6 or DFT_TC_TF32X3
  int K = 0, J = 0;
  int npad = 0;               // MMA N: K rounded up to a multiple of 16
  int nchunk_f = 0;           // reduction chunks, forward (K)
  int nchunk_i = 0;           // reduction chunks, inverse (2J)
  const unsigned char* bf = nullptr;  // forward matrix pieces, shared-memory core layout per chunk
  const unsigned char* bi = nullptr;  // inverse matrix pieces
  int* err = nullptr;         // device flag: nonzero after a bounded wait gave up
  size_t chunk_bytes = 0;     // bytes of all pieces of one chunk of the matrix
  bool stall_next = false;    // test hook: the next launch's first barrier waits for 16 bytes never sent
};

// Host side: sizes of the matrix tables for K time steps and a scheme.
size_t dft_tc_table_bytes(int K, int scheme, bool inverse);
// Host side: fill the forward / inverse tables (FP64 entries, split into pieces).
void dft_tc_build_table(int K, int scheme, bool inverse, unsigned char* out);
// Chunk geometry of the tables.
void dft_tc_geometry(int K, int scheme, DftTc* d);

// x: FP64 [K][nblk] time slices -> X: complex FP32 [J][nblk].
void launch_dft_tc_forward(DftTc& d, long long nblk, const double* x, cpx<float>* X, cudaStream_t st);
// X: complex FP32 [J][nblk] -> y: FP64 [K][nblk].
void launch_dft_tc_inverse(DftTc& d, long long nblk, const cpx<float>* X, double* y, cudaStream_t st);

}  // namespace pint
