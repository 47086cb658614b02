// k_dft_tc.cu -- the time DFT of the FP32 preconditioner as a dense real
// contraction on the 5th-generation tensor cores.
//
// One CTA per SM, persistent over tiles of TC_M = 128 spatial slots.  For a
// tile, D[128][npad] (FP32, tensor memory) = A[128][Kred] * B[Kred][npad]:
// A holds the tile's input (FP64 time slices, or FP32 complex frequency
// values) split into BF16 or TF32 pieces by the CTA's threads and stored in
// shared memory in the K-major no-swizzle core-matrix layout; B is the
// constant DFT matrix, pre-split and pre-laid-out on the host, brought in by
// bulk asynchronous copies (cp.async.bulk) per reduction chunk of TC_KC.
// One elected thread issues tcgen05.mma for every kept piece product and
// commits to an mbarrier per pipeline stage; two stages overlap the next
// chunk's loads with the current chunk's MMAs.  The leading (hi x hi)
// products accumulate in D1 (TMEM columns 0..255) and the correction
// products in D2 (columns 256..511), summed in the epilogue: the large sum
// then takes one FP32 accumulation per MMA step instead of one per product.  The epilogue reads the
// accumulator with tcgen05.ld (warp w reads TMEM lanes 32 (w mod 4) + lane,
// i.e. one spatial slot per thread) and writes coalesced rows of the output.
//
// Every mbarrier wait is bounded (one second of global time); a wait
// that gives up sets *err, the CTA waits (bounded) for its own MMAs and bulk
// copies in flight, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <string.h>

#include <cmath>
#include <vector>

#include "dft_tc.h"

namespace pint {
namespace {

constexpr int TC_M = 128;           // spatial slots per tile (TMEM lanes)
constexpr int TC_KC = 32;           // reduction elements per pipeline chunk
constexpr int TC_THREADS = 256;
constexpr int TC_STAGES = 2;
constexpr uint32_t TC_TMEM_COLS = 512;
constexpr uint32_t TC_D2 = 256;     // column of the second accumulator
constexpr unsigned long long TC_WAIT_NS = 1000000000ull;  // 1 s of global time

template <int S>
struct Scheme;
// three BF16 pieces per operand; products (0,0) (0,1) (1,0) (0,2) (1,1) (2,0)
template <>
struct Scheme<DFT_TC_BF16X6> {
  static constexpr int ESZ = 2;
  static constexpr int NP = 3;
  static constexpr int NPROD = 6;
  static constexpr uint32_t FMT = 1;  // instruction-descriptor operand format: BF16
  __host__ __device__ static constexpr int pa(int p) { return p == 0 ? 0 : p == 1 ? 0 : p == 2 ? 1 : p == 3 ? 0 : p == 4 ? 1 : 2; }
  __host__ __device__ static constexpr int pb(int p) { return p == 0 ? 0 : p == 1 ? 1 : p == 2 ? 0 : p == 3 ? 2 : p == 4 ? 1 : 0; }
};
// two TF32 pieces per operand; products (0,0) (0,1) (1,0)
template <>
struct Scheme<DFT_TC_TF32X3> {
  static constexpr int ESZ = 4;
  static constexpr int NP = 2;
  static constexpr int NPROD = 3;
  static constexpr uint32_t FMT = 2;  // TF32
  __host__ __device__ static constexpr int pa(int p) { return p == 2 ? 1 : 0; }
  __host__ __device__ static constexpr int pb(int p) { return p == 1 ? 1 : 0; }
};

// Byte geometry of one operand piece (rows x TC_KC reduction elements):
// core matrices of 8 rows x 16 bytes stored as 128 contiguous bytes; cores
// adjacent along the reduction are LBO = 128 bytes apart, 8-row groups are
// SBO = (TC_KC * esz / 16) * 128 bytes apart.
__host__ __device__ constexpr int core_cols(int esz) { return TC_KC * esz / 16; }
__host__ __device__ constexpr int sbo_bytes(int esz) { return core_cols(esz) * 128; }
__host__ __device__ inline size_t core_offset(int row, int kk, int esz) {
  return (size_t)(row >> 3) * sbo_bytes(esz) + (size_t)((kk * esz) >> 4) * 128 + (size_t)(row & 7) * 16 +
         (size_t)((kk * esz) & 15);
}

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for the phase of the given parity; false if it gave up
__device__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try(bar, parity)) return true;
    if (global_ns() - t0 > TC_WAIT_NS) return false;
  }
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(cols) : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
}
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);  // descriptor version 1, base offset 0, no swizzle
}
template <int S>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (S == DFT_TC_BF16X6) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  }
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// 16 consecutive 32-bit accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v);
// Columns col .. col+15 of the accumulator at column `base`, reading no column
// at or beyond base + limit (the block is shifted back and realigned; values
// past the limit come back as 0).  col is warp-uniform.
__device__ __forceinline__ void tmem_ld16_lim(uint32_t tl, uint32_t base, int col, int limit, float* v) {
  if (col + 16 <= limit) {
    tmem_ld16(tl + base + (uint32_t)col, v);
    return;
  }
  const int cs = limit - 16, shift = col - cs;
  float t[16];
  tmem_ld16(tl + base + (uint32_t)cs, t);
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    float val = 0.f;
#pragma unroll
    for (int s2 = 0; s2 < 16; ++s2)
      if (s2 == shift && q + s2 < 16) val = t[q + s2];
    v[q] = val;
  }
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// ---------------------------------------------------------------- operand splitting
__device__ __forceinline__ uint32_t tf32_rna(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ uint16_t bf16_rn(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }
__device__ __forceinline__ float bf16_f(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

// 16 consecutive reduction values of one row -> NP pieces, stored as 16-byte
// core rows at their place in the stage's A pieces.
template <int S>
__device__ __forceinline__ void store_split(unsigned char* a_base, size_t piece_bytes, int row, int kk0,
                                            const float* v) {
  using Sc = Scheme<S>;
  if constexpr (S == DFT_TC_BF16X6) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {  // two core columns of 8 values
      uint32_t w[3][4];
#pragma unroll
      for (int e = 0; e < 8; e += 2) {
        uint16_t h[2], m[2], l[2];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          const float x = v[c * 8 + e + t];
          h[t] = bf16_rn(x);
          const float r1 = x - bf16_f(h[t]);
          m[t] = bf16_rn(r1);
          l[t] = bf16_rn(r1 - bf16_f(m[t]));
        }
        w[0][e / 2] = (uint32_t)h[0] | ((uint32_t)h[1] << 16);
        w[1][e / 2] = (uint32_t)m[0] | ((uint32_t)m[1] << 16);
        w[2][e / 2] = (uint32_t)l[0] | ((uint32_t)l[1] << 16);
      }
      const size_t off = core_offset(row, kk0 + c * 8, Sc::ESZ);
#pragma unroll
      for (int p = 0; p < 3; ++p)
        *reinterpret_cast<uint4*>(a_base + p * piece_bytes + off) = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
    }
  } else {
#pragma unroll
    for (int c = 0; c < 4; ++c) {  // four core columns of 4 values
      uint32_t h[4], l[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float x = v[c * 4 + e];
        h[e] = tf32_rna(x);
        l[e] = tf32_rna(x - __uint_as_float(h[e]));
      }
      const size_t off = core_offset(row, kk0 + c * 4, Sc::ESZ);
      *reinterpret_cast<uint4*>(a_base + off) = make_uint4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<uint4*>(a_base + piece_bytes + off) = make_uint4(l[0], l[1], l[2], l[3]);
    }
  }
}

struct TcArgs {
  int K, J, npad, nchunk;
  long long nblk;
  const double* x;       // forward input  [K][nblk]
  cpx<float>* X;         // forward output [J][nblk]
  const cpx<float>* Xi;  // inverse input  [J][nblk]
  double* y;             // inverse output [K][nblk]
  const unsigned char* table;
  size_t chunk_bytes;
  int* err;
  unsigned extra_tx;  // test hook: bytes the first chunk's barrier expects beyond its copy (0 normally)
};

template <int S>
__host__ __device__ constexpr size_t a_piece_bytes() {
  return (size_t)TC_M * TC_KC * Scheme<S>::ESZ;
}

template <int S, int DIR>
__global__ void __launch_bounds__(TC_THREADS, 1) dft_tc_kernel(TcArgs a) {
  using Sc = Scheme<S>;
  extern __shared__ __align__(1024) unsigned char smem[];
  constexpr size_t APB = a_piece_bytes<S>();
  constexpr size_t ABYTES = APB * Sc::NP;
  const size_t stage_bytes = ABYTES + a.chunk_bytes;
  const size_t bpb = a.chunk_bytes / Sc::NP;  // bytes of one B piece
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + TC_STAGES * stage_bytes);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2 * TC_STAGES);
  int* abort_flag = reinterpret_cast<int*>(tslot + 1);
  const uint32_t bbar0 = smem_u32(bars), mbar0 = smem_u32(bars + TC_STAGES);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(bbar0 + 8 * s, 1);
      mbar_init(mbar0 + 8 * s, 1);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(smem_u32(tslot), TC_TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  const uint32_t idesc = (1u << 4) | (Sc::FMT << 7) | (Sc::FMT << 10) | ((uint32_t)(a.npad >> 3) << 17) |
                         ((uint32_t)(TC_M >> 4) << 24);
  constexpr uint32_t LBO = 128, SBO = sbo_bytes(Sc::ESZ);
  constexpr int STEPS = TC_KC * Sc::ESZ / 32;  // MMAs (32 reduction bytes each) per chunk and product

  const long long ntiles = (a.nblk + TC_M - 1) / TC_M;
  const int row = tid & (TC_M - 1), half = tid >> 7;
  unsigned g = 0;  // chunks issued by this CTA (all tiles)
  bool ok = true;
  int cm[TC_STAGES] = {0, 0}, cb[TC_STAGES] = {0, 0};  // commits / bulk copies issued per stage

  for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const long long col = tile * TC_M + row;
    const bool in = col < a.nblk;
    for (int ch = 0; ch < a.nchunk; ++ch, ++g) {
      const int s = g & 1;
      unsigned char* st = smem + s * stage_bytes;
      bool fail = false;
      // the MMAs that last read this stage must be done
      if (g >= 2 && !mbar_wait(mbar0 + 8 * s, ((g >> 1) - 1) & 1)) fail = true;
      if (__syncthreads_or(fail)) {
        ok = false;
        break;
      }
      if (tid == 0) {
        mbar_arrive_tx(bbar0 + 8 * s, (uint32_t)a.chunk_bytes + (g == 0 ? a.extra_tx : 0u));
        bulk_g2s(smem_u32(st + ABYTES), a.table + (size_t)ch * a.chunk_bytes, (uint32_t)a.chunk_bytes,
                 bbar0 + 8 * s);
        ++cb[s];
      }
      // this thread's 16 reduction values of the chunk
      float v[16];
      const int kk0 = half * 16;
      const int c0 = ch * TC_KC + kk0;
      if (DIR == 0) {
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = (in && c0 + q < a.K) ? (float)__ldg(a.x + (size_t)(c0 + q) * a.nblk + col) : 0.f;
      } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int j = (c0 >> 1) + q;
          float2 z = make_float2(0.f, 0.f);
          if (in && j < a.J) z = __ldg(reinterpret_cast<const float2*>(a.Xi) + (size_t)j * a.nblk + col);
          v[2 * q] = z.x;
          v[2 * q + 1] = z.y;
        }
      }
      store_split<S>(st, APB, row, kk0, v);
      fence_proxy_async();
      if (tid == 0 && !mbar_wait(bbar0 + 8 * s, ((g >> 1)) & 1)) fail = true;
      if (__syncthreads_or(fail)) {
        ok = false;
        break;
      }
      if (tid == 0) {
        tc_fence_after();
        const uint32_t abase = smem_u32(st), bbase = smem_u32(st + ABYTES);
#pragma unroll
        for (int p = 0; p < Sc::NPROD; ++p)
#pragma unroll
          for (int t = 0; t < STEPS; ++t) {
            const uint64_t ad = smem_desc(abase + (uint32_t)(Sc::pa(p) * APB) + 256u * t, LBO, SBO);
            const uint64_t bd = smem_desc(bbase + (uint32_t)(Sc::pb(p) * bpb) + 256u * t, LBO, SBO);
            // leading product (hi x hi) into D1 (columns 0..), the smaller
            // correction products into D2 (columns 256..): the FP32 sums of
            // the large terms then take one accumulation per MMA step only
            if (p == 0)
              mma<S>(tmem, ad, bd, idesc, (ch > 0 || t > 0) ? 1u : 0u);
            else
              mma<S>(tmem + TC_D2, ad, bd, idesc, (ch > 0 || p > 1 || t > 0) ? 1u : 0u);
          }
        mma_commit(mbar0 + 8 * s);
        ++cm[s];
      }
    }
    if (!ok) break;
    // accumulator complete once the last chunk's commit has arrived
    {
      const unsigned gl = g - 1;
      bool fail = !mbar_wait(mbar0 + 8 * (gl & 1), (gl >> 1) & 1);
      if (__syncthreads_or(fail)) {
        ok = false;
        break;
      }
    }
    tc_fence_after();
    const int lg = warp & 3, grp = warp >> 2;
    const uint32_t tl = tmem + ((uint32_t)(32 * lg) << 16);
    const long long i = tile * TC_M + 32 * lg + lane;
    float re[16], im[16], c2[16];
    constexpr int LIM = (int)TC_D2;  // columns per accumulator
    if (DIR == 0) {
      const int Jh = (a.J + 1) / 2;
      const int j0 = grp * Jh, j1 = min(a.J, j0 + Jh);
      for (int jb = j0; jb < j1; jb += 16) {
        tmem_ld16_lim(tl, 0, jb, LIM, re);
        tmem_ld16_lim(tl, TC_D2, jb, LIM, c2);
#pragma unroll
        for (int q = 0; q < 16; ++q) re[q] += c2[q];
        tmem_ld16_lim(tl, 0, a.J - 1 + jb, LIM, im);
        tmem_ld16_lim(tl, TC_D2, a.J - 1 + jb, LIM, c2);
#pragma unroll
        for (int q = 0; q < 16; ++q) im[q] += c2[q];
        if (i < a.nblk)
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int j = jb + q;
            if (j < j1) {
              const float vi = (j >= 1 && j <= a.K - a.J) ? im[q] : 0.f;
              a.X[(size_t)j * a.nblk + i] = mkc<float>(re[q], vi);
            }
          }
      }
    } else {
      const int Kh = (a.K + 1) / 2;
      const int k0 = grp * Kh, k1 = min(a.K, k0 + Kh);
      for (int kb = k0; kb < k1; kb += 16) {
        tmem_ld16_lim(tl, 0, kb, LIM, re);
        tmem_ld16_lim(tl, TC_D2, kb, LIM, c2);
        if (i < a.nblk)
#pragma unroll
          for (int q = 0; q < 16; ++q)
            if (kb + q < k1) a.y[(size_t)(kb + q) * a.nblk + i] = (double)re[q] + (double)c2[q];
      }
    }
    tc_fence_before();
    __syncthreads();
  }

  if (!ok) {
    // a bounded wait gave up: record it, let this CTA's MMAs and bulk copies
    // in flight finish (bounded), then release the tensor memory
    if (tid == 0) {
      atomicExch(a.err, 1);
      for (int s = 0; s < TC_STAGES; ++s) {
        if (cm[s] > 0) mbar_wait(mbar0 + 8 * s, (cm[s] - 1) & 1);
        if (cb[s] > 0) mbar_wait(bbar0 + 8 * s, (cb[s] - 1) & 1);
      }
    }
    tc_fence_before();
    __syncthreads();
  }
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, TC_TMEM_COLS);
}

// ---------------------------------------------------------------- host tables
uint16_t host_bf16(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);  // round to nearest even (finite inputs)
  return (uint16_t)(u >> 16);
}
double host_bf16_val(uint16_t b) {
  const uint32_t u = (uint32_t)b << 16;
  float f;
  memcpy(&f, &u, 4);
  return f;
}
uint32_t host_tf32(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  return (u + 0x1000u) & 0xFFFFE000u;  // round to nearest, ties away from zero
}
double host_tf32_val(uint32_t b) {
  float f;
  memcpy(&f, &b, 4);
  return f;
}

int esz_of(int scheme) { return scheme == DFT_TC_BF16X6 ? 2 : 4; }
int np_of(int scheme) { return scheme == DFT_TC_BF16X6 ? 3 : 2; }

}  // namespace

void dft_tc_geometry(int K, int scheme, DftTc* d) {
  d->scheme = scheme;
  d->K = K;
  d->J = K / 2 + 1;
  d->npad = (K + 15) / 16 * 16;
  d->nchunk_f = (K + TC_KC - 1) / TC_KC;
  d->nchunk_i = (2 * d->J + TC_KC - 1) / TC_KC;
  d->chunk_bytes = (size_t)np_of(scheme) * d->npad * TC_KC * esz_of(scheme);
}

size_t dft_tc_table_bytes(int K, int scheme, bool inverse) {
  DftTc d;
  dft_tc_geometry(K, scheme, &d);
  return d.chunk_bytes * (inverse ? d.nchunk_i : d.nchunk_f);
}

void dft_tc_build_table(int K, int scheme, bool inverse, unsigned char* out) {
  DftTc d;
  dft_tc_geometry(K, scheme, &d);
  const int J = d.J, esz = esz_of(scheme), np = np_of(scheme);
  const int nchunk = inverse ? d.nchunk_i : d.nchunk_f;
  const size_t piece = (size_t)d.npad * TC_KC * esz;
  memset(out, 0, d.chunk_bytes * nchunk);
  const double two_pi = 2.0 * M_PI;
  for (int o = 0; o < K; ++o)
    for (int c = 0; c < nchunk * TC_KC; ++c) {
      double v = 0.0;
      if (!inverse) {
        if (c < K) v = o < J ? std::cos(two_pi * (double)(((long long)o * c) % K) / K)
                             : -std::sin(two_pi * (double)(((long long)(o - J + 1) * c) % K) / K);
      } else {
        const int j = c / 2;
        if (j < J) {
          const double w = (j == 0 || 2 * j == K) ? 1.0 : 2.0;
          const double ang = two_pi * (double)(((long long)j * o) % K) / K;
          v = w / K * ((c & 1) ? -std::sin(ang) : std::cos(ang));
        }
      }
      if (v == 0.0) continue;
      unsigned char* chunk = out + (size_t)(c / TC_KC) * d.chunk_bytes;
      const size_t off = core_offset(o, c % TC_KC, esz);
      if (scheme == DFT_TC_BF16X6) {
        const uint16_t h = host_bf16((float)v);
        const double r1 = v - host_bf16_val(h);
        const uint16_t m = host_bf16((float)r1);
        const uint16_t l = host_bf16((float)(r1 - host_bf16_val(m)));
        const uint16_t pcs[3] = {h, m, l};
        for (int p = 0; p < np; ++p) memcpy(chunk + p * piece + off, &pcs[p], 2);
      } else {
        const uint32_t h = host_tf32((float)v);
        const uint32_t l = host_tf32((float)(v - host_tf32_val(h)));
        memcpy(chunk + off, &h, 4);
        memcpy(chunk + piece + off, &l, 4);
      }
    }
}

namespace {
template <int S, int DIR>
void launch_tc(const DftTc& d, const TcArgs& a, cudaStream_t st) {
  // SM count of the device, queried once (thread-safe initialisation)
  static const int nsm = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
  }();
  const size_t stage = a_piece_bytes<S>() * Scheme<S>::NP + d.chunk_bytes;
  size_t smem = TC_STAGES * stage + 2 * TC_STAGES * 8 + 16;
  // at least 116 KB so that one CTA (and one 512-column TMEM allocation) fits per SM
  if (smem < 116 * 1024) smem = 116 * 1024;
  cudaFuncSetAttribute(dft_tc_kernel<S, DIR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const long long ntiles = (a.nblk + TC_M - 1) / TC_M;
  const int grid = (int)(ntiles < nsm ? ntiles : nsm);
  if (grid <= 0) return;
  dft_tc_kernel<S, DIR><<<grid, TC_THREADS, smem, st>>>(a);
}
}  // namespace

void launch_dft_tc_forward(DftTc& d, long long nblk, const double* x, cpx<float>* X, cudaStream_t st) {
  TcArgs a{d.K, d.J, d.npad, d.nchunk_f, nblk, x, X, nullptr, nullptr, d.bf, d.chunk_bytes, d.err,
           d.stall_next ? 16u : 0u};
  if (d.scheme == DFT_TC_BF16X6)
    launch_tc<DFT_TC_BF16X6, 0>(d, a, st);
  else
    launch_tc<DFT_TC_TF32X3, 0>(d, a, st);
  d.stall_next = false;
}

void launch_dft_tc_inverse(DftTc& d, long long nblk, const cpx<float>* X, double* y, cudaStream_t st) {
  TcArgs a{d.K, d.J, d.npad, d.nchunk_i, nblk, nullptr, nullptr, X, y, d.bi, d.chunk_bytes, d.err,
           d.stall_next ? 16u : 0u};
  if (d.scheme == DFT_TC_BF16X6)
    launch_tc<DFT_TC_BF16X6, 1>(d, a, st);
  else
    launch_tc<DFT_TC_TF32X3, 1>(d, a, st);
  d.stall_next = false;
}

}  // namespace pint
