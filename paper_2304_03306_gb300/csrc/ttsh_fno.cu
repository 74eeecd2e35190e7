// ttsh_fno.cu - learned corrector: a Fourier neural operator (FNO) that corrects a coarse,
// 4x-larger-time-step solver step, with forward and backward kernels for training on the GPU.
//
// The network (Li et al., ICLR 2021): lift (Cin -> C, bias), L Fourier layers
//   z = h W + b + SpectralConv(h),  h' = GELU(z) (no GELU after the last layer),
// and a projection C -> 1.  SpectralConv = irfft2(P(W_modes * P^T(rfft2(h)))) keeping kx < m
// and ky in {0..m-1} U {n-m..n-1}, one complex C x C matrix per kept mode.
//
// Arithmetic: learned weights are held as FP32 master copies and used in BF16 by the kernels;
// every product accumulates in FP32.  The channel-mixing layers (h W, and dz W^T in the
// backward pass) run on the 5th-generation tensor cores (tcgen05.mma BF16 -> FP32 in tensor
// memory, fused bias / residual / GELU epilogue).  The transforms restricted to the kept
// modes are exact DFT matrices (2m x n per row and per column, cheaper than a full FFT when
// m << n).  The row transforms (onto the kept kx and back, and their adjoints in the backward
// pass) run on the tensor cores as well (BF16 operands, FP32 accumulation); the column
// transforms along y with the per-mode complex mixing run in dedicated FP32 kernels that read
// BF16 weights.
// Gradients use fixed-order partial sums, so repeated calls give identical bits.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ttsh.h"
#include "ttsh_ops.h"
#include "ttsh_wait.cuh"

namespace fno_dev {

// ---------------------------------------------------------------------------------------
// FP32 batched GEMM: C[b] = alpha * op(A[b]) * op(B[b]) + beta * C[b] (row-major, 64x64 tiles)
// ---------------------------------------------------------------------------------------
struct Gemm {
  int M, N, K, batch;
  const float* A;
  long long lda, sA;
  const float* B;
  long long ldb, sB;
  float* C;
  long long ldc, sC;
  float alpha, beta;
};

template <bool TA, bool TB>
__global__ void __launch_bounds__(256) sgemm_kernel(Gemm g) {
  __shared__ float As[16][64 + 4];
  __shared__ float Bs[16][64 + 4];
  const long long bz = blockIdx.z;
  const float* A = g.A + bz * g.sA;
  const float* B = g.B + bz * g.sB;
  float* C = g.C + bz * g.sC;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = 0; k0 < g.K; k0 += 16) {
    for (int e = threadIdx.x; e < 1024; e += 256) {
      int mm, kk;
      if (TA) { mm = e & 63; kk = e >> 6; } else { kk = e & 15; mm = e >> 4; }
      const int m = m0 + mm, k = k0 + kk;
      float v = 0.f;
      if (m < g.M && k < g.K) v = TA ? A[(long long)k * g.lda + m] : A[(long long)m * g.lda + k];
      As[kk][mm] = v;
    }
    for (int e = threadIdx.x; e < 1024; e += 256) {
      int nn, kk;
      if (TB) { kk = e & 15; nn = e >> 4; } else { nn = e & 63; kk = e >> 6; }
      const int n = n0 + nn, k = k0 + kk;
      float v = 0.f;
      if (n < g.N && k < g.K) v = TB ? B[(long long)n * g.ldb + k] : B[(long long)k * g.ldb + n];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + 16 * i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx + 16 * j;
      if (n >= g.N) continue;
      float* c = C + (long long)m * g.ldc + n;
      const float prev = g.beta != 0.f ? g.beta * *c : 0.f;
      *c = g.alpha * acc[i][j] + prev;
    }
  }
}

cudaError_t sgemm(bool ta, bool tb, int M, int N, int K, int batch, float alpha, const float* A,
                  long long lda, long long sA, const float* B, long long ldb, long long sB, float beta,
                  float* C, long long ldc, long long sC, cudaStream_t s) {
  Gemm g{M, N, K, batch, A, lda, sA, B, ldb, sB, C, ldc, sC, alpha, beta};
  dim3 grid((N + 63) / 64, (M + 63) / 64, batch);
  if (ta && tb) sgemm_kernel<true, true><<<grid, 256, 0, s>>>(g);
  else if (ta) sgemm_kernel<true, false><<<grid, 256, 0, s>>>(g);
  else if (tb) sgemm_kernel<false, true><<<grid, 256, 0, s>>>(g);
  else sgemm_kernel<false, false><<<grid, 256, 0, s>>>(g);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Tensor-core channel mixing: out[p][o] = sum_i A[p][i] Bt[o][i] (+ epilogue), C = 32
// ---------------------------------------------------------------------------------------
constexpr int CW = 32;   // width the tensor-core kernels are written for

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

enum { EPI_FWD = 0, EPI_FWD_LAST = 1, EPI_BWD = 2 };

struct PwArgs {
  const __nv_bfloat16* A;   // P x 32
  const __nv_bfloat16* Bt;  // 32 x 32, [o][i]
  const float* bias;        // 32 (forward) or nullptr
  const float* add;         // P x 32 residual added to the product
  float* out;               // P x 32: z (forward) or dh (backward)
  float* h;                 // P x 32: GELU(z) (forward)
  __nv_bfloat16* hb;        // P x 32: GELU(z) in BF16 (forward)
  long long P;
  int* err;                 // set to 1 if a tensor-core completion wait ran out
};

// ---------------------------------------------------------------------------------------
// Channel mixing on the 5th-generation tensor cores (tcgen05).  A CTA of 4 warps owns a
// 128 x 32 FP32 accumulator in tensor memory; per 128-row tile it stages A (128 x 32 BF16)
// in shared memory in the canonical K-major layout without swizzle (8-row x 16-byte core
// matrices, K-adjacent core matrices 128 B apart, row groups 512 B apart), one thread issues
// two tcgen05.mma (M = 128, N = 32, K = 16 each; B = the 32 x 32 weight, staged once), the
// completion is signalled on an mbarrier by tcgen05.commit, and each warp reads its 32
// accumulator lanes with tcgen05.ld for the fused bias / residual / GELU epilogue.  Every
// wait is bounded: on time-out the CTA records the error, releases its tensor memory and
// returns.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading (K) and stride (M/N) byte offsets,
// descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

constexpr int kTcRows = 128;

// (r, k) of a 128 x 32 (or 32 x 32) BF16 K-major tile -> byte offset in the core-matrix layout
__device__ __forceinline__ int core_off(int r, int kc) { return (r >> 3) * 512 + kc * 128 + (r & 7) * 16; }

template <int EPI>
__global__ void __launch_bounds__(128) pointwise_tc_kernel(PwArgs a) {
  __shared__ __align__(1024) uint8_t sa[kTcRows * CW * 2];
  __shared__ __align__(1024) uint8_t sb[CW * CW * 2];
  __shared__ float sbias[CW];
  __shared__ float stile[4 * 32 * 33];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int c = tid; c < CW * 4; c += 128) {
    const int r = c >> 2, kc = c & 3;
    *reinterpret_cast<uint4*>(sb + core_off(r, kc)) = *reinterpret_cast<const uint4*>(a.Bt + r * CW + kc * 8);
  }
  if (tid < CW) sbias[tid] = (EPI != EPI_BWD) ? a.bias[tid] : 0.f;
  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)) : "memory");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(&tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const long long ntiles = (a.P + kTcRows - 1) / kTcRows;
  uint32_t phase = 0;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const long long row0 = t * kTcRows;
    for (int c = tid; c < kTcRows * 4; c += 128) {
      const int r = c >> 2, kc = c & 3;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (row0 + r < a.P) v = *reinterpret_cast<const uint4*>(a.A + (row0 + r) * CW + kc * 8);
      *reinterpret_cast<uint4*>(sa + core_off(r, kc)) = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> tensor core
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      constexpr uint32_t id = umma_idesc_bf16(kTcRows, CW);
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        const uint64_t ad = umma_desc(smem_u32(sa) + ks * 256, 128, 512);
        const uint64_t bd = umma_desc(smem_u32(sb) + ks * 256, 128, 512);
        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                     ::"r"(tmem), "l"(ad), "l"(bd), "r"(id), "r"(ks) : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   ::"r"(smem_u32(&mbar)) : "memory");
    }
    const bool done = ttsh::mbar_wait_bounded(smem_u32(&mbar), phase, ttsh::kWaitLimitNs);
    if (__syncthreads_or(!done)) {
      if (tid == 0) atomicExch(a.err, 1);
      break;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    uint32_t r[CW];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                   "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                   "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(tmem + ((uint32_t)(warp * 32) << 16)));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    // Epilogue through a padded 32 x 33 shared tile per warp: the warp's 32 rows are one
    // contiguous 4 KB block in global memory, so the residual is read and the results are
    // written with consecutive lanes on consecutive addresses; each thread then works on its
    // own row (the accumulator layout) without bank conflicts.
    float* tile = stile + warp * 32 * 33;
    const long long p0 = row0 + warp * 32;
    const int nrows = a.P - p0 >= 32 ? 32 : (a.P - p0 > 0 ? (int)(a.P - p0) : 0);
    for (int j = 0; j < nrows; ++j) tile[j * 33 + lane] = a.add[(p0 + j) * CW + lane];
    __syncwarp();
    float v[CW];
#pragma unroll
    for (int o = 0; o < CW; ++o) {
      v[o] = __uint_as_float(r[o]) + tile[lane * 33 + o];
      if (EPI != EPI_BWD) v[o] += sbias[o];
    }
    __syncwarp();
    if (a.out) {
#pragma unroll
      for (int o = 0; o < CW; ++o) tile[lane * 33 + o] = v[o];
      __syncwarp();
      for (int j = 0; j < nrows; ++j) a.out[(p0 + j) * CW + lane] = tile[j * 33 + lane];
      __syncwarp();
    }
    if (EPI != EPI_BWD) {
#pragma unroll
      for (int o = 0; o < CW; ++o) tile[lane * 33 + o] = EPI == EPI_FWD ? gelu(v[o]) : v[o];
      __syncwarp();
      if (a.h)
        for (int j = 0; j < nrows; ++j) a.h[(p0 + j) * CW + lane] = tile[j * 33 + lane];
      if (EPI == EPI_FWD && a.hb) {
        // two rows per warp instruction: lanes 0-15 row j, 16-31 row j + 1, two channels each
        const int half = lane >> 4, c2 = (lane & 15) * 2;
        for (int j = half; j < nrows; j += 2)
          *reinterpret_cast<__nv_bfloat162*>(a.hb + (p0 + j) * CW + c2) =
              __floats2bfloat162_rn(tile[j * 33 + c2], tile[j * 33 + c2 + 1]);
      }
      __syncwarp();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");   // accumulator read before reuse
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem) : "memory");
}

// ---------------------------------------------------------------------------------------
// Restricted row transforms on the tensor cores.  With q = (sample, y) a grid row and the 32
// channels c, the four row contractions of a spectral layer are
//   contract over x:  out[q][j][c] = sum_x M[j][x] act[q][x][c]   (row DFT onto the kept kx,
//                     and the adjoint of the inverse row transform)
//   expand to x:      out[q][x][c] = sum_j M[x][j] in[q][j][c]    (inverse row transform onto
//                     the grid, and the adjoint of the row DFT)
// with j over the 2m <= 32 kept (Re, Im) kx entries.  Both are tcgen05.mma kind::f16 with
// BF16 operands staged in shared memory in the canonical K-major layout without swizzle
// (8-row x 16-byte core matrices; K-adjacent core matrices 128 B apart, 8-row groups
// K * 16 B apart) and a 128 x 32 FP32 accumulator per MMA group in tensor memory.
//   contract: M = 128 rows (4 grid rows x 32 channels), N = 32 (j, padded), K = n (x);
//             the activation tile is transposed into the K-major layout while it is staged.
//   expand:   M = 128 x values of one x tile, N = 32 channels, K = 32 (j, padded); the CTA
//             keeps its x tile of M and walks over grid rows two at a time (two accumulators).
// Completion is an mbarrier signalled by tcgen05.commit with a bounded wait (time-out: error
// word, tensor memory released, CTA returns).
// ---------------------------------------------------------------------------------------
struct XcArgs {
  const __nv_bfloat16* M;     // contract: [32][n] (rows j >= J zero); expand: [n][32] (columns j >= J zero)
  const __nv_bfloat16* act;   // contract: [Q][n][32] BF16
  const float* in;            // expand:   [Q][J][32] FP32 (rounded to BF16 when staged)
  float* out;                 // contract: [Q][J][32]; expand: [Q][n][32]
  int n, J;
  long long Q;
  int* err;
};

__device__ __forceinline__ void tc_alloc(uint32_t* dst, int cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(cols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t tmem, int cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols) : "memory");
}
__device__ __forceinline__ void tc_mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t id, int accumulate) {
  asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
               "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
               ::"r"(tmem), "l"(ad), "l"(bd), "r"(id), "r"(accumulate) : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 32 accumulator columns of this warp's 32 lanes
__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
               "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
               "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                 "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                 "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                 "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

constexpr int kXcMaxN = 512;
inline int xcontract_smem(int n) { return 128 * n * 2 + 32 * n * 2 + 128; }

__global__ void __launch_bounds__(128) xcontract_tc_kernel(XcArgs a) {
  extern __shared__ __align__(16) uint8_t xc_dyn[];
  uint8_t* sa = xc_dyn + ((128u - (smem_u32(xc_dyn) & 127u)) & 127u);   // 128 x n activation tile
  uint8_t* sb = sa + 128 * a.n * 2;                                      // 32 x n matrix
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = a.n, nk = n >> 3, SBO = n * 16;
  for (int c = tid; c < 32 * nk; c += 128) {
    const int r = c / nk, kc = c % nk;
    *reinterpret_cast<uint4*>(sb + (r >> 3) * SBO + kc * 128 + (r & 7) * 16) =
        *reinterpret_cast<const uint4*>(a.M + (long long)r * n + kc * 8);
  }
  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)) : "memory");
  if (warp == 0) tc_alloc(&tmem_base, 32);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const long long ntiles = (a.Q + 3) / 4;
  uint32_t phase = 0;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const long long q0 = t * 4;
    // activation tile, transposed: row m = 32 qi + c, column k = x <- act[q0 + qi][x][c]
    // (16-byte loads of 8 channels, eight 2-byte stores into one core-matrix column)
    // (eight loads in flight per thread before their stores; 16 n units of 8 channels)
    for (int u0 = tid; u0 < 4 * n * 4; u0 += 8 * 128) {
      uint4 v[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int u = u0 + i * 128, x = (u >> 2) % n, qi = (u >> 2) / n;
        v[i] = make_uint4(0, 0, 0, 0);
        if (u < 16 * n && q0 + qi < a.Q)
          v[i] = *reinterpret_cast<const uint4*>(a.act + ((q0 + qi) * n + x) * CW + (u & 3) * 8);
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int u = u0 + i * 128, c8 = u & 3, x = (u >> 2) % n, qi = (u >> 2) / n;
        if (u >= 16 * n) break;   // past the tile (n not a multiple of 64)
        const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&v[i]);
        uint8_t* dst = sa + (qi * 4 + c8) * SBO + (x >> 3) * 128 + (x & 7) * 2;
#pragma unroll
        for (int k = 0; k < 8; ++k) *reinterpret_cast<__nv_bfloat16*>(dst + k * 16) = e[k];
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> tensor core
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      constexpr uint32_t id = umma_idesc_bf16(kTcRows, CW);
      for (int ks = 0; ks < n / 16; ++ks)
        tc_mma_bf16(tmem, umma_desc(smem_u32(sa) + ks * 256, 128, SBO), umma_desc(smem_u32(sb) + ks * 256, 128, SBO),
                    id, ks);
      tc_commit(&mbar);
    }
    const bool done = ttsh::mbar_wait_bounded(smem_u32(&mbar), phase, ttsh::kWaitLimitNs);
    if (__syncthreads_or(!done)) {
      if (tid == 0) atomicExch(a.err, 1);
      break;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    uint32_t r[CW];
    tc_ld32(tmem + ((uint32_t)(warp * 32) << 16), r);
    const long long q = q0 + warp;   // this warp's accumulator rows: grid row q0 + warp, channel = lane
    if (q < a.Q)
      for (int j = 0; j < a.J; ++j) a.out[(q * a.J + j) * CW + lane] = __uint_as_float(r[j]);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, 32);
}

__global__ void __launch_bounds__(128) xexpand_tc_kernel(XcArgs a) {
  __shared__ __align__(1024) uint8_t sa[128 * 32 * 2];       // 128 x 32 matrix tile
  __shared__ __align__(1024) uint8_t sbt[2 * 32 * 32 * 2];   // two 32 (c) x 32 (j) operands
  __shared__ float stile[4 * 32 * 33];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = a.n, x0 = blockIdx.x * 128;
  for (int c = tid; c < 128 * 4; c += 128) {
    const int r = c >> 2, kc = c & 3;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (x0 + r < n) v = *reinterpret_cast<const uint4*>(a.M + (long long)(x0 + r) * 32 + kc * 8);
    *reinterpret_cast<uint4*>(sa + core_off(r, kc)) = v;
  }
  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)) : "memory");
  if (warp == 0) tc_alloc(&tmem_base, 64);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const long long npairs = (a.Q + 1) / 2;
  uint32_t phase = 0;
  for (long long pr = blockIdx.y; pr < npairs; pr += gridDim.y) {
    const long long q0 = pr * 2;
    // operands: row c, column k = j <- in[q0 + qi][j][c] (zero for j >= J or past the end)
    for (int u = tid; u < 2 * 32 * 32; u += 128) {
      const int c = u & 31, j = (u >> 5) & 31, qi = u >> 10;
      float v = 0.f;
      if (j < a.J && q0 + qi < a.Q) v = a.in[((q0 + qi) * a.J + j) * CW + c];
      *reinterpret_cast<__nv_bfloat16*>(sbt + qi * 2048 + core_off(c, j >> 3) + (j & 7) * 2) = __float2bfloat16_rn(v);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      constexpr uint32_t id = umma_idesc_bf16(kTcRows, CW);
      for (int qi = 0; qi < 2; ++qi)
        for (int ks = 0; ks < 2; ++ks)
          tc_mma_bf16(tmem + qi * 32, umma_desc(smem_u32(sa) + ks * 256, 128, 512),
                      umma_desc(smem_u32(sbt) + qi * 2048 + ks * 256, 128, 512), id, ks);
      tc_commit(&mbar);
    }
    const bool done = ttsh::mbar_wait_bounded(smem_u32(&mbar), phase, ttsh::kWaitLimitNs);
    if (__syncthreads_or(!done)) {
      if (tid == 0) atomicExch(a.err, 1);
      break;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // epilogue: this warp's 32 x rows of each grid row, through a padded 32 x 33 tile so that
    // the stores are 128-byte rows of consecutive channels
    float* tile = stile + warp * 32 * 33;
    const int xw = x0 + warp * 32;
    const int nrows = n - xw >= 32 ? 32 : (n - xw > 0 ? n - xw : 0);
    for (int qi = 0; qi < 2; ++qi) {
      uint32_t r[CW];
      tc_ld32(tmem + ((uint32_t)(warp * 32) << 16) + qi * 32, r);
      const long long q = q0 + qi;
      if (q >= a.Q) continue;
#pragma unroll
      for (int c = 0; c < CW; ++c) tile[lane * 33 + c] = __uint_as_float(r[c]);
      __syncwarp();
      for (int i = 0; i < nrows; ++i) a.out[(q * n + xw + i) * CW + lane] = tile[i * 33 + lane];
      __syncwarp();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, 64);
}

// ---------------------------------------------------------------------------------------
// Elementwise kernels
// ---------------------------------------------------------------------------------------
// h0 = x Wp + bp (Cin inputs), FP32 and BF16 copies
__global__ void lift_kernel(const float* __restrict__ x, const float* __restrict__ Wp, const float* __restrict__ bp,
                            int cin, long long P, float* __restrict__ h, __nv_bfloat16* __restrict__ hb) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P * CW) return;
  const long long p = i / CW;
  const int c = (int)(i % CW);
  float acc = bp[c];
  for (int k = 0; k < cin; ++k) acc = fmaf(x[p * cin + k], Wp[k * CW + c], acc);
  h[i] = acc;
  hb[i] = __float2bfloat16_rn(acc);
}

// out[p] = h[p] . Wq + bq; with a target: dout = 2 (out - t) / npts, dh = dout Wq, and
// per-block partial sums of (out - t)^2
__global__ void __launch_bounds__(256) project_kernel(const float* __restrict__ h, const float* __restrict__ Wq,
                                                      const float* __restrict__ bq, long long P, float* __restrict__ out,
                                                      const float* __restrict__ target, float* __restrict__ dout,
                                                      float* __restrict__ dh, double* __restrict__ lpart) {
  __shared__ double red[256];
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double sq = 0.0;
  if (p < P) {
    float acc = bq[0];
#pragma unroll
    for (int c = 0; c < CW; ++c) acc = fmaf(h[p * CW + c], Wq[c], acc);
    out[p] = acc;
    if (target) {
      const float r = acc - target[p];
      sq = (double)r * r;
      const float g = 2.f * r / (float)P;
      dout[p] = g;
#pragma unroll
      for (int c = 0; c < CW; ++c) dh[p * CW + c] = g * Wq[c];
    }
  }
  if (!target) return;
  red[threadIdx.x] = sq;
  __syncthreads();
  for (int s = 128; s >= 1; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) lpart[blockIdx.x] = red[0];
}

// dz = dh * GELU'(z) (FP32 and BF16); for the last layer (no GELU) dz = dh
__global__ void gelu_bwd_kernel(const float* __restrict__ dh, const float* __restrict__ z, long long n, int act,
                                float* __restrict__ dz, __nv_bfloat16* __restrict__ dzb) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float v = act ? dh[i] * gelu_grad(z[i]) : dh[i];
  dz[i] = v;
  dzb[i] = __float2bfloat16_rn(v);
}

// Partial weight gradients over a chunk of points: part[blk][i*cd + o] = sum_p A[p][i] D[p][o],
// part[blk][ca*cd + o] = sum_p D[p][o]  (ca, cd <= 32; fixed order)
__global__ void __launch_bounds__(256) wgrad_partial_kernel(const float* __restrict__ A, int ca,
                                                            const float* __restrict__ D, int cd, long long P,
                                                            int chunk, float* __restrict__ part) {
  __shared__ float As[64][33];
  __shared__ float Ds[64][33];
  const int nout = ca * cd + cd;
  float acc[5] = {0, 0, 0, 0, 0};   // up to 5 outputs per thread (1056 / 256 -> 5)
  const long long p0 = (long long)blockIdx.x * chunk;
  const long long p1 = p0 + chunk < P ? p0 + chunk : P;
  for (long long pb = p0; pb < p1; pb += 64) {
    for (int e = threadIdx.x; e < 64 * 32; e += 256) {
      const int r = e >> 5, c = e & 31;
      const long long p = pb + r;
      As[r][c] = (p < p1 && c < ca) ? A[p * ca + c] : 0.f;
      Ds[r][c] = (p < p1 && c < cd) ? D[p * cd + c] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const int o = threadIdx.x + 256 * q;
      if (o < nout) {
        const int i = o / cd, j = o % cd;
        float s = 0.f;
        if (i < ca)
          for (int r = 0; r < 64; ++r) s = fmaf(As[r][i], Ds[r][j], s);
        else
          for (int r = 0; r < 64; ++r) s += Ds[r][j];
        acc[q] += s;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const int o = threadIdx.x + 256 * q;
    if (o < nout) part[(long long)blockIdx.x * nout + o] = acc[q];
  }
}

// grad[w_off + i*cd + o] = sum_blk part (then bias at b_off + o); fixed order over blocks
__global__ void wgrad_reduce_kernel(const float* __restrict__ part, int nblk, int ca, int cd,
                                    float* __restrict__ gw, float* __restrict__ gb) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  const int nout = ca * cd + cd;
  if (o >= nout) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[(long long)b * nout + o];
  if (o < ca * cd) gw[o] = (float)s;
  else gb[o - ca * cd] = (float)s;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}

// Row DFT onto the kept kx for one (sample, y) row: Hx[k][c] = sum_x F[k][x] h[x][c], with
// F rows 0..m-1 = cos, m..2m-1 = -sin (2 pi kx x / n).  One block of 256 threads per row.
__global__ void __launch_bounds__(256) row_dft_kernel(const float* __restrict__ h, const float* __restrict__ F,
                                                      int n, int m, float* __restrict__ Hx) {
  extern __shared__ __align__(16) float sm[];
  float* hs = sm;            // [n][C]
  float* fs = sm + n * CW;   // [2m][n]
  const long long q = blockIdx.x;
  const float* hq = h + q * n * CW;
  for (int e = threadIdx.x; e < n * CW / 4; e += 256) cp_async16(hs + 4 * e, hq + 4 * e);
  for (int e = threadIdx.x; e < 2 * m * n / 4; e += 256) cp_async16(fs + 4 * e, F + 4 * e);
  asm volatile("cp.async.commit_group;\ncp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  // thread (c, g) computes kx rows k = g, g + 8, ...; four x at a time from float4 loads
  const int c = threadIdx.x % CW, g = threadIdx.x / CW;
  for (int k0 = g; k0 < 2 * m; k0 += 32) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int x = 0; x < n; x += 4) {
      const float h0 = hs[x * CW + c], h1 = hs[(x + 1) * CW + c], h2 = hs[(x + 2) * CW + c], h3 = hs[(x + 3) * CW + c];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int k = k0 + 8 * r;
        if (k < 2 * m) {
          const float4 fv = *reinterpret_cast<const float4*>(fs + k * n + x);
          acc[r] = fmaf(fv.x, h0, fmaf(fv.y, h1, fmaf(fv.z, h2, fmaf(fv.w, h3, acc[r]))));
        }
      }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int k = k0 + 8 * r;
      if (k < 2 * m) Hx[(q * 2 * m + k) * CW + c] = acc[r];
    }
  }
}

// Inverse row transform for one (sample, y) row: s[x][c] = sum_k Bx[x][k] Z[k][c] over the
// 2m kept (Re, Im) kx entries; each thread keeps its channel's Z column in registers.
constexpr int MAXJ = 64;
__global__ void __launch_bounds__(256) row_idft_kernel(const float* __restrict__ Z, const float* __restrict__ Bx,
                                                       int n, int m, float* __restrict__ sout) {
  extern __shared__ __align__(16) float bs[];   // [n][2m]
  const long long q = blockIdx.x;
  const int J = 2 * m;
  for (int e = threadIdx.x; e < n * J / 4; e += 256) cp_async16(bs + 4 * e, Bx + 4 * e);
  asm volatile("cp.async.commit_group;\ncp.async.wait_all;\n" ::: "memory");
  const int c = threadIdx.x % CW, g = threadIdx.x / CW;
  float z[MAXJ];
#pragma unroll
  for (int k = 0; k < MAXJ; ++k) z[k] = k < J ? Z[(q * J + k) * CW + c] : 0.f;
  __syncthreads();
  for (int x = g; x < n; x += 8) {
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < MAXJ; k += 4) {
      if (k < J) {
        const float4 bv = *reinterpret_cast<const float4*>(bs + x * J + k);
        acc = fmaf(bv.x, z[k], fmaf(bv.y, z[k + 1], fmaf(bv.z, z[k + 2], fmaf(bv.w, z[k + 3], acc))));
      }
    }
    sout[(q * n + x) * CW + c] = acc;
  }
}

inline int row_idft_smem(int n, int m) { return n * 2 * m * 4; }

inline int row_dft_smem(int n, int m) { return (n * CW + 2 * m * n) * 4; }

// Column-local part of a spectral layer, for one (sample b, kx), in two kernels so that the
// work spreads over many blocks (there are only m kx values per sample):
//   column_fwd_mix_kernel, grid (kx, b, 2m/JB): H[j][c] = sum_y G[j][y] X[y][c] for JB kept ky
//     rows (X = the row-DFT output column, G = exp(-2 pi i ky_j y / n)), written to global for
//     the backward pass, then Y[j][o] = sum_i W[j][kx][i][o] H[j][i] (BF16 weights, FP32 sums);
//   column_inv_kernel, grid (kx, b, n/YB): Z[y][c] = sum_j conj(G[j][y]) Y[j][c] for YB rows,
//     stored as the Re | Im halves of each (b, y) row that the inverse row transform reads.
constexpr int JB = 4, YB = 16;

__global__ void __launch_bounds__(JB * CW) column_fwd_mix_kernel(
    const float* __restrict__ Hx, const float* __restrict__ Gr, const float* __restrict__ Gi,
    const __nv_bfloat16* __restrict__ Wr, const __nv_bfloat16* __restrict__ Wi, int n, int m,
    float* __restrict__ Hr_out, float* __restrict__ Hi_out, float* __restrict__ Yr_out, float* __restrict__ Yi_out) {
  extern __shared__ __align__(16) float sm[];
  const int kx = blockIdx.x, b = blockIdx.y, j0 = blockIdx.z * JB, tid = threadIdx.x;
  const int J = 2 * m;
  const long long mC = (long long)m * CW, rowstride = 2 * mC;
  float* xr = sm;
  float* xi = xr + n * CW;
  float* gr = xi + n * CW;     // [JB][n]
  float* gi = gr + JB * n;
  float* hr = gi + JB * n;     // [JB][C]
  float* hi = hr + JB * CW;
  const float* xb = Hx + (long long)b * n * rowstride + (long long)kx * CW;
  for (int e = tid; e < n * (CW / 4); e += JB * CW) {
    const int y = e / (CW / 4), c4 = (e % (CW / 4)) * 4;
    cp_async16(xr + y * CW + c4, xb + (long long)y * rowstride + c4);
    cp_async16(xi + y * CW + c4, xb + (long long)y * rowstride + mC + c4);
  }
  for (int e = tid; e < JB * n / 4; e += JB * CW) {
    cp_async16(gr + 4 * e, Gr + (long long)j0 * n + 4 * e);
    cp_async16(gi + 4 * e, Gi + (long long)j0 * n + 4 * e);
  }
  asm volatile("cp.async.commit_group;\ncp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  const int c = tid % CW, jl = tid / CW, j = j0 + jl;
  float ar = 0.f, ai = 0.f;
#pragma unroll 8
  for (int y = 0; y < n; ++y) {
    const float a = gr[jl * n + y], bb = gi[jl * n + y];
    const float u = xr[y * CW + c], v = xi[y * CW + c];
    ar = fmaf(a, u, fmaf(-bb, v, ar));
    ai = fmaf(a, v, fmaf(bb, u, ai));
  }
  hr[jl * CW + c] = ar;
  hi[jl * CW + c] = ai;
  const long long o = (((long long)b * J + j) * m + kx) * CW + c;
  Hr_out[o] = ar;
  Hi_out[o] = ai;
  __syncwarp();
  const __nv_bfloat16* wr = Wr + ((long long)j * m + kx) * CW * CW;
  const __nv_bfloat16* wi = Wi + ((long long)j * m + kx) * CW * CW;
  float yr = 0.f, yi = 0.f;
#pragma unroll 16
  for (int i = 0; i < CW; ++i) {
    const float a = __bfloat162float(wr[i * CW + c]), bb = __bfloat162float(wi[i * CW + c]);
    const float u = hr[jl * CW + i], v = hi[jl * CW + i];
    yr = fmaf(a, u, fmaf(-bb, v, yr));
    yi = fmaf(a, v, fmaf(bb, u, yi));
  }
  Yr_out[o] = yr;
  Yi_out[o] = yi;
}

__global__ void __launch_bounds__(256) column_inv_kernel(const float* __restrict__ Yr, const float* __restrict__ Yi,
                                                         const float* __restrict__ Gr, const float* __restrict__ Gi,
                                                         int n, int m, float* __restrict__ Z) {
  __shared__ float yr[64][CW], yi[64][CW];
  const int kx = blockIdx.x, b = blockIdx.y, y0 = blockIdx.z * YB, tid = threadIdx.x;
  const int J = 2 * m;
  const long long mC = (long long)m * CW, rowstride = 2 * mC;
  for (int e = tid; e < J * CW; e += 256) {
    const int j = e / CW, c = e % CW;
    const long long o = (((long long)b * J + j) * m + kx) * CW + c;
    yr[j][c] = Yr[o];
    yi[j][c] = Yi[o];
  }
  __syncthreads();
  const int c = tid % CW;
  float* zb = Z + (long long)b * n * rowstride + (long long)kx * CW;
  for (int yl = tid / CW; yl < YB; yl += 256 / CW) {
    const int y = y0 + yl;
    float ar = 0.f, ai = 0.f;
    for (int j = 0; j < J; ++j) {   // conj(G[j][y]) = Gr - i Gi
      const float a = Gr[(long long)j * n + y], bb = -Gi[(long long)j * n + y];
      ar = fmaf(a, yr[j][c], fmaf(-bb, yi[j][c], ar));
      ai = fmaf(a, yi[j][c], fmaf(bb, yr[j][c], ai));
    }
    zb[(long long)y * rowstride + c] = ar;
    zb[(long long)y * rowstride + mC + c] = ai;
  }
}

inline int column_fwd_mix_smem(int n) { return (2 * n * CW + 2 * JB * n + 2 * JB * CW) * 4; }


// Mode mixing, forward: Y[b][mode][o] = sum_i W[mode][i][o] H[b][mode][i] (complex, BF16 weights)
__global__ void __launch_bounds__(CW) modemix_fwd_kernel(const float* __restrict__ Hr, const float* __restrict__ Hi,
                                                         const __nv_bfloat16* __restrict__ Wr,
                                                         const __nv_bfloat16* __restrict__ Wi, int nmodes, int B,
                                                         float* __restrict__ Yr, float* __restrict__ Yi) {
  __shared__ float wr[CW][CW + 1], wi[CW][CW + 1], hr[CW], hi[CW];
  const int mode = blockIdx.x, o = threadIdx.x;
  for (int i = 0; i < CW; ++i) {
    wr[i][o] = __bfloat162float(Wr[((long long)mode * CW + i) * CW + o]);
    wi[i][o] = __bfloat162float(Wi[((long long)mode * CW + i) * CW + o]);
  }
  for (int b = 0; b < B; ++b) {
    const long long base = ((long long)b * nmodes + mode) * CW;
    __syncthreads();
    hr[o] = Hr[base + o];
    hi[o] = Hi[base + o];
    __syncthreads();
    float yr = 0.f, yi = 0.f;
    for (int i = 0; i < CW; ++i) {
      yr = fmaf(wr[i][o], hr[i], fmaf(-wi[i][o], hi[i], yr));
      yi = fmaf(wr[i][o], hi[i], fmaf(wi[i][o], hr[i], yi));
    }
    Yr[base + o] = yr;
    Yi[base + o] = yi;
  }
}

// Mode mixing, backward: dH = W^H dY per mode; dW[i][o] = sum_b dY_o conj(H_i)
__global__ void __launch_bounds__(256) modemix_bwd_kernel(const float* __restrict__ Hr, const float* __restrict__ Hi,
                                                          const float* __restrict__ dYr, const float* __restrict__ dYi,
                                                          const __nv_bfloat16* __restrict__ Wr,
                                                          const __nv_bfloat16* __restrict__ Wi, int nmodes, int B,
                                                          float* __restrict__ dHr, float* __restrict__ dHi,
                                                          float* __restrict__ gWr, float* __restrict__ gWi) {
  __shared__ float wr[CW][CW + 1], wi[CW][CW + 1];
  __shared__ float hr[CW], hi[CW], yr[CW], yi[CW];
  const int mode = blockIdx.x, tid = threadIdx.x;
  for (int e = tid; e < CW * CW; e += 256) {
    const int i = e / CW, o = e % CW;
    wr[i][o] = __bfloat162float(Wr[(long long)mode * CW * CW + e]);
    wi[i][o] = __bfloat162float(Wi[(long long)mode * CW * CW + e]);
  }
  float ar[4] = {0, 0, 0, 0}, ai[4] = {0, 0, 0, 0};
  for (int b = 0; b < B; ++b) {
    const long long base = ((long long)b * nmodes + mode) * CW;
    __syncthreads();
    if (tid < CW) {
      hr[tid] = Hr[base + tid];
      hi[tid] = Hi[base + tid];
      yr[tid] = dYr[base + tid];
      yi[tid] = dYi[base + tid];
    }
    __syncthreads();
    if (tid < CW) {   // dH_i = sum_o conj(W_io) dY_o
      const int i = tid;
      float sr = 0.f, si = 0.f;
      for (int o = 0; o < CW; ++o) {
        sr = fmaf(wr[i][o], yr[o], fmaf(wi[i][o], yi[o], sr));
        si = fmaf(wr[i][o], yi[o], fmaf(-wi[i][o], yr[o], si));
      }
      dHr[base + i] = sr;
      dHi[base + i] = si;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + 256 * q;
      const int i = e / CW, o = e % CW;
      ar[q] = fmaf(yr[o], hr[i], fmaf(yi[o], hi[i], ar[q]));
      ai[q] = fmaf(yi[o], hr[i], fmaf(-yr[o], hi[i], ai[q]));
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int e = tid + 256 * q;
    gWr[(long long)mode * CW * CW + e] = ar[q];
    gWi[(long long)mode * CW * CW + e] = ai[q];
  }
}

// Adam with bias correction on the FP32 master weights
__global__ void adam_kernel(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void to_bf16_kernel(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = __float2bfloat16_rn(src[i]);
}

// W (32x32, [i][o]) -> BF16 copies of W^T ([o][i], forward operand) and W ([i][o], backward)
__global__ void pointwise_weights_kernel(const float* __restrict__ W, __nv_bfloat16* __restrict__ Wt,
                                         __nv_bfloat16* __restrict__ Wn) {
  const int e = threadIdx.x + blockIdx.x * blockDim.x;
  if (e >= CW * CW) return;
  const int i = e / CW, o = e % CW;
  Wt[o * CW + i] = __float2bfloat16_rn(W[e]);
  Wn[e] = __float2bfloat16_rn(W[e]);
}

// Input channels of sample b from a domain's staging (omega, v_x, v_y as doubles) and K
template <typename T>
__global__ void features_kernel(const double* __restrict__ real, const T* __restrict__ K, long long nn,
                                float s0, float s1, float s2, float s3, float* __restrict__ x) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nn) return;
  x[p * 4 + 0] = (float)real[p] * s0;
  x[p * 4 + 1] = (float)real[nn + p] * s1;
  x[p * 4 + 2] = (float)real[2 * nn + p] * s2;
  x[p * 4 + 3] = (float)K[p] * s3;
}

__global__ void diff_kernel(const double* __restrict__ a, const double* __restrict__ b, long long n, float scale,
                            float* __restrict__ out) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) out[p] = (float)(a[p] - b[p]) * scale;
}

__global__ void to_double_scaled_kernel(const float* __restrict__ src, long long n, float scale,
                                        double* __restrict__ dst) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) dst[p] = (double)src[p] * (double)scale;
}

}  // namespace fno_dev

// =======================================================================================
// Host side
// =======================================================================================
using namespace fno_dev;

struct ttsh_fno {
  ttsh_fno_config cfg;
  cudaStream_t stream;
  int n, C, m, L, cin, Bmax;
  long long nn, Pmax;
  long long nparams;
  // parameter offsets (floats) in the flat vector, same order as the host layout
  long long off_Wp, off_bp, off_Wq, off_bq;
  std::vector<long long> off_Wr, off_Wi, off_W, off_b;
  float *theta = nullptr, *grad = nullptr, *adam_m = nullptr, *adam_v = nullptr;
  __nv_bfloat16* wbf = nullptr;                 // BF16 copies: per layer Wr, Wi (spectral), Wt, Wn
  std::vector<long long> boff_Wr, boff_Wi, boff_Wt, boff_Wn;
  // DFT matrices
  float *Fx = nullptr, *Gr = nullptr, *Gi = nullptr, *Gpr = nullptr, *Gpi = nullptr, *Bx = nullptr;
  // activations
  std::vector<float*> h, z;                     // h[0..L], z[0..L-1]
  std::vector<__nv_bfloat16*> hb;               // hb[0..L-1]
  std::vector<float*> Hr, Hi;                   // kept input modes per layer
  float *Hx = nullptr, *Yr = nullptr, *Yi = nullptr, *Z = nullptr, *s = nullptr;
  float *dh = nullptr, *dz = nullptr, *dspec = nullptr, *dout = nullptr, *yo = nullptr;
  __nv_bfloat16* dzb = nullptr;
  float *wpart = nullptr;
  double* lpart = nullptr;
  int* tc_err = nullptr;        // set by the tensor-core kernels when a completion wait ran out
  int wchunk, nwblk;
  float in_scale[4] = {1, 1, 1, 1}, out_scale = 1;
  bool fused_columns = false;   // row_dft / column kernels fit in shared memory
  // BF16 matrices of the row contractions on the tensor cores (tc_rows: n % 16 == 0,
  // n <= 512, 2m <= 32): Fx [32][n], Bx [n][32], Fx^T [n][32], Bx^T [32][n], zero-padded
  __nv_bfloat16 *FxB = nullptr, *BxB = nullptr, *FxTB = nullptr, *BxTB = nullptr;
  bool tc_rows = false;
  long long adam_t = 0;
  std::vector<void*> allocs;
};

namespace {

ttsh_status fno_fail(ttsh_status st, const char* msg) {
  ttsh::set_last_error(msg);
  return st;
}

ttsh_status fno_cuda(cudaError_t e, const char* what) {
  ttsh::set_last_error(what, e);
  return TTSH_E_CUDA;
}

#define FNO_CUDA(call, what)                        \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return fno_cuda(e_, what); \
  } while (0)

// Grid of the tensor-core kernels: one CTA per 128-row tile, at most 4 resident per SM.
unsigned tc_grid(long long P) {
  const long long tiles = (P + kTcRows - 1) / kTcRows;
  return (unsigned)(tiles < 152 * 4 ? tiles : 152 * 4);
}

// out[q][j][c] = sum_x M[j][x] act[q][x][c] on the tensor cores (Q grid rows)
cudaError_t run_xcontract(ttsh_fno* f, const __nv_bfloat16* M, const __nv_bfloat16* act, long long Q, float* out) {
  XcArgs a{M, act, nullptr, out, f->n, 2 * f->m, Q, f->tc_err};
  const long long tiles = (Q + 3) / 4;
  const unsigned grid = (unsigned)(tiles < 152 * 2 ? tiles : 152 * 2);
  xcontract_tc_kernel<<<grid, 128, xcontract_smem(f->n), f->stream>>>(a);
  return cudaGetLastError();
}

// out[q][x][c] = sum_j M[x][j] in[q][j][c] on the tensor cores
cudaError_t run_xexpand(ttsh_fno* f, const __nv_bfloat16* M, const float* in, long long Q, float* out) {
  XcArgs a{M, nullptr, in, out, f->n, 2 * f->m, Q, f->tc_err};
  const int xt = (f->n + 127) / 128;
  const long long pairs = (Q + 1) / 2;
  const long long per = (152LL * 6) / xt;
  dim3 grid((unsigned)xt, (unsigned)(pairs < per ? pairs : per));
  xexpand_tc_kernel<<<grid, 128, 0, f->stream>>>(a);
  return cudaGetLastError();
}

// Report (once) a tensor-core completion wait that ran out; called at synchronising entries.
ttsh_status check_tc(ttsh_fno* f) {
  int h = 0;
  FNO_CUDA(cudaMemcpyAsync(&h, f->tc_err, sizeof(int), cudaMemcpyDeviceToHost, f->stream), "read tensor-core status");
  FNO_CUDA(cudaStreamSynchronize(f->stream), "read tensor-core status");
  if (h) {
    FNO_CUDA(cudaMemsetAsync(f->tc_err, 0, sizeof(int), f->stream), "clear tensor-core status");
    return fno_fail(TTSH_E_TIMEOUT, "a tensor-core completion wait ran out");
  }
  return TTSH_OK;
}

template <typename P>
cudaError_t dalloc(ttsh_fno* f, P** ptr, size_t bytes) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e == cudaSuccess) {
    f->allocs.push_back(p);
    *ptr = static_cast<P*>(p);
  }
  return e;
}

// SplitMix64 (Steele, Lea & Flood 2014), output i of the stream from `seed`
uint64_t sm64(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
double u01(uint64_t seed, uint64_t i) { return (double)(sm64(seed, i) >> 11) * (1.0 / 9007199254740992.0); }

cudaError_t refresh_bf16(ttsh_fno* f) {
  cudaStream_t s = f->stream;
  const long long msz = (long long)2 * f->m * f->m * f->C * f->C;
  for (int l = 0; l < f->L; ++l) {
    to_bf16_kernel<<<(unsigned)((msz + 255) / 256), 256, 0, s>>>(f->theta + f->off_Wr[l], f->wbf + f->boff_Wr[l], msz);
    to_bf16_kernel<<<(unsigned)((msz + 255) / 256), 256, 0, s>>>(f->theta + f->off_Wi[l], f->wbf + f->boff_Wi[l], msz);
    pointwise_weights_kernel<<<(CW * CW + 255) / 256, 256, 0, s>>>(f->theta + f->off_W[l], f->wbf + f->boff_Wt[l],
                                                                    f->wbf + f->boff_Wn[l]);
  }
  return cudaGetLastError();
}

// Forward pass for B samples (x: B*n*n x cin); leaves activations for backward.
ttsh_status forward_impl(ttsh_fno* f, const float* x, int B, float* out, const float* target, double* loss) {
  cudaStream_t s = f->stream;
  const int n = f->n, C = f->C, m = f->m, L = f->L;
  const long long P = (long long)B * f->nn;
  const long long mC = (long long)m * C;
  const int nmodes = 2 * m * m;
  lift_kernel<<<(unsigned)((P * C + 255) / 256), 256, 0, s>>>(x, f->theta + f->off_Wp, f->theta + f->off_bp,
                                                              f->cin, P, f->h[0], f->hb[0]);
  for (int l = 0; l < L; ++l) {
    const float* hl = f->h[l];
    // row DFT: Hx[q] (2m x C) = Fx (2m x n) . h[q] (n x C), q = (b, y)
    if (f->tc_rows) {
      FNO_CUDA(run_xcontract(f, f->FxB, f->hb[l], (long long)B * n, f->Hx), "row DFT (tensor cores)");
    } else if (f->fused_columns) {
      row_dft_kernel<<<(unsigned)(B * n), 256, row_dft_smem(n, m), s>>>(hl, f->Fx, n, m, f->Hx);
      FNO_CUDA(cudaGetLastError(), "row DFT");
    } else {
      FNO_CUDA(sgemm(false, false, 2 * m, C, n, B * n, 1.f, f->Fx, n, 0, hl, C, (long long)n * C, 0.f, f->Hx, C,
                     2LL * m * C, s), "row DFT");
    }
    const long long sX = (long long)n * 2 * mC, sH = 2LL * m * mC;
    if (f->fused_columns) {
      // column DFT + mode mixing (JB ky rows per block), then inverse column DFT (YB rows per block)
      column_fwd_mix_kernel<<<dim3(m, B, 2 * m / JB), JB * CW, column_fwd_mix_smem(n), s>>>(
          f->Hx, f->Gr, f->Gi, f->wbf + f->boff_Wr[l], f->wbf + f->boff_Wi[l], n, m, f->Hr[l], f->Hi[l], f->Yr, f->Yi);
      column_inv_kernel<<<dim3(m, B, n / YB), 256, 0, s>>>(f->Yr, f->Yi, f->Gr, f->Gi, n, m, f->Z);
      FNO_CUDA(cudaGetLastError(), "spectral column kernels");
    } else {
      // column DFT per sample: H = G X (complex), X = Hx_b viewed as n x 2mC
      FNO_CUDA(sgemm(false, false, 2 * m, (int)mC, n, B, 1.f, f->Gr, n, 0, f->Hx, 2 * mC, sX, 0.f, f->Hr[l], mC, sH, s), "col DFT");
      FNO_CUDA(sgemm(false, false, 2 * m, (int)mC, n, B, -1.f, f->Gi, n, 0, f->Hx + mC, 2 * mC, sX, 1.f, f->Hr[l], mC, sH, s), "col DFT");
      FNO_CUDA(sgemm(false, false, 2 * m, (int)mC, n, B, 1.f, f->Gr, n, 0, f->Hx + mC, 2 * mC, sX, 0.f, f->Hi[l], mC, sH, s), "col DFT");
      FNO_CUDA(sgemm(false, false, 2 * m, (int)mC, n, B, 1.f, f->Gi, n, 0, f->Hx, 2 * mC, sX, 1.f, f->Hi[l], mC, sH, s), "col DFT");
      // mode mixing
      modemix_fwd_kernel<<<nmodes, CW, 0, s>>>(f->Hr[l], f->Hi[l], f->wbf + f->boff_Wr[l], f->wbf + f->boff_Wi[l],
                                               nmodes, B, f->Yr, f->Yi);
      // inverse column: Z (n x mC complex, stored as Re | Im blocks of width mC) = G' Y
      FNO_CUDA(sgemm(false, false, n, (int)mC, 2 * m, B, 1.f, f->Gpr, 2 * m, 0, f->Yr, mC, sH, 0.f, f->Z, 2 * mC, sX, s), "inv col");
      FNO_CUDA(sgemm(false, false, n, (int)mC, 2 * m, B, -1.f, f->Gpi, 2 * m, 0, f->Yi, mC, sH, 1.f, f->Z, 2 * mC, sX, s), "inv col");
      FNO_CUDA(sgemm(false, false, n, (int)mC, 2 * m, B, 1.f, f->Gpr, 2 * m, 0, f->Yi, mC, sH, 0.f, f->Z + mC, 2 * mC, sX, s), "inv col");
      FNO_CUDA(sgemm(false, false, n, (int)mC, 2 * m, B, 1.f, f->Gpi, 2 * m, 0, f->Yr, mC, sH, 1.f, f->Z + mC, 2 * mC, sX, s), "inv col");
    }
    // inverse row: s[q] (n x C) = Bx (n x 2m) . Z[q] (2m x C)
    if (f->tc_rows) {
      FNO_CUDA(run_xexpand(f, f->BxB, f->Z, (long long)B * n, f->s), "inverse row (tensor cores)");
    } else if (f->fused_columns) {
      row_idft_kernel<<<(unsigned)(B * n), 256, row_idft_smem(n, m), s>>>(f->Z, f->Bx, n, m, f->s);
      FNO_CUDA(cudaGetLastError(), "inv row");
    } else {
      FNO_CUDA(sgemm(false, false, n, C, 2 * m, B * n, 1.f, f->Bx, 2 * m, 0, f->Z, C, 2LL * m * C, 0.f, f->s, C,
                     (long long)n * C, s), "inv row");
    }
    // z = h W + b + s on the tensor cores, then GELU
    PwArgs a;
    a.A = f->hb[l];
    a.Bt = f->wbf + f->boff_Wt[l];
    a.bias = f->theta + f->off_b[l];
    a.add = f->s;
    a.out = target ? f->z[l] : nullptr;   // pre-activations are kept only for the backward pass
    a.h = f->h[l + 1];
    a.hb = l + 1 < L ? f->hb[l + 1] : nullptr;
    a.P = P;
    a.err = f->tc_err;
    const unsigned nblk = tc_grid(P);
    if (l + 1 < L) pointwise_tc_kernel<EPI_FWD><<<nblk, 128, 0, s>>>(a);
    else pointwise_tc_kernel<EPI_FWD_LAST><<<nblk, 128, 0, s>>>(a);
    FNO_CUDA(cudaGetLastError(), "pointwise layer");
  }
  const unsigned pblk = (unsigned)((P + 255) / 256);
  project_kernel<<<pblk, 256, 0, s>>>(f->h[L], f->theta + f->off_Wq, f->theta + f->off_bq, P, out, target,
                                      f->dout, f->dh, f->lpart);
  FNO_CUDA(cudaGetLastError(), "projection");
  if (target && loss) {
    std::vector<double> lp(pblk);
    FNO_CUDA(cudaMemcpyAsync(lp.data(), f->lpart, pblk * sizeof(double), cudaMemcpyDeviceToHost, s), "loss");
    FNO_CUDA(cudaStreamSynchronize(s), "loss");
    double acc = 0;
    for (double v : lp) acc += v;
    *loss = acc / (double)P;
  }
  return TTSH_OK;
}

ttsh_status wgrad(ttsh_fno* f, const float* A, int ca, const float* D, int cd, long long P, float* gw, float* gb) {
  const int nout = ca * cd + cd;
  const long long chunk = (P + f->nwblk - 1) / f->nwblk;
  const int nblk = (int)((P + chunk - 1) / chunk);
  wgrad_partial_kernel<<<nblk, 256, 0, f->stream>>>(A, ca, D, cd, P, (int)chunk, f->wpart);
  wgrad_reduce_kernel<<<(nout + 255) / 256, 256, 0, f->stream>>>(f->wpart, nblk, ca, cd, gw, gb);
  FNO_CUDA(cudaGetLastError(), "weight gradient");
  return TTSH_OK;
}

ttsh_status backward_impl(ttsh_fno* f, const float* x, int B, const float* out) {
  cudaStream_t s = f->stream;
  const int n = f->n, C = f->C, m = f->m, L = f->L;
  const long long P = (long long)B * f->nn;
  const long long mC = (long long)m * C;
  const long long sX = (long long)n * 2 * mC, sH = 2LL * m * mC;
  const int nmodes = 2 * m * m;
  (void)out;
  ttsh_status st;
  // projection: dWq = h_L^T dout, dbq = sum dout; dh (= dout Wq) was written by project_kernel
  if ((st = wgrad(f, f->h[L], C, f->dout, 1, P, f->grad + f->off_Wq, f->grad + f->off_bq)) != TTSH_OK) return st;
  for (int l = L - 1; l >= 0; --l) {
    const long long tot = P * C;
    gelu_bwd_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(f->dh, f->z[l], tot, l + 1 < L ? 1 : 0, f->dz, f->dzb);
    FNO_CUDA(cudaGetLastError(), "gelu backward");
    if ((st = wgrad(f, f->h[l], C, f->dz, C, P, f->grad + f->off_W[l], f->grad + f->off_b[l])) != TTSH_OK) return st;
    // spectral adjoint: dZ[q] = Bx^T dz[q]
    if (f->tc_rows) {
      FNO_CUDA(run_xcontract(f, f->BxTB, f->dzb, (long long)B * n, f->Z), "inv row adjoint (tensor cores)");
    } else {
      FNO_CUDA(sgemm(true, false, 2 * m, C, n, B * n, 1.f, f->Bx, 2 * m, 0, f->dz, C, (long long)n * C, 0.f, f->Z, C,
                     2LL * m * C, s), "inv row adjoint");
    }
    // dY = G'^H dZ
    FNO_CUDA(sgemm(true, false, 2 * m, (int)mC, n, B, 1.f, f->Gpr, 2 * m, 0, f->Z, 2 * mC, sX, 0.f, f->Yr, mC, sH, s), "inv col adjoint");
    FNO_CUDA(sgemm(true, false, 2 * m, (int)mC, n, B, 1.f, f->Gpi, 2 * m, 0, f->Z + mC, 2 * mC, sX, 1.f, f->Yr, mC, sH, s), "inv col adjoint");
    FNO_CUDA(sgemm(true, false, 2 * m, (int)mC, n, B, 1.f, f->Gpr, 2 * m, 0, f->Z + mC, 2 * mC, sX, 0.f, f->Yi, mC, sH, s), "inv col adjoint");
    FNO_CUDA(sgemm(true, false, 2 * m, (int)mC, n, B, -1.f, f->Gpi, 2 * m, 0, f->Z, 2 * mC, sX, 1.f, f->Yi, mC, sH, s), "inv col adjoint");
    // mode mixing adjoint (dH into Hx-sized scratch halves) and spectral weight gradients
    float* dHr = f->s;                         // reuse: 2*m*mC*B floats each
    float* dHi = f->s + (long long)B * sH;
    modemix_bwd_kernel<<<nmodes, 256, 0, s>>>(f->Hr[l], f->Hi[l], f->Yr, f->Yi, f->wbf + f->boff_Wr[l],
                                              f->wbf + f->boff_Wi[l], nmodes, B, dHr, dHi, f->grad + f->off_Wr[l],
                                              f->grad + f->off_Wi[l]);
    FNO_CUDA(cudaGetLastError(), "mode mixing adjoint");
    // dX = G^H dH (written as Re | Im blocks into Hx)
    FNO_CUDA(sgemm(true, false, n, (int)mC, 2 * m, B, 1.f, f->Gr, n, 0, dHr, mC, sH, 0.f, f->Hx, 2 * mC, sX, s), "col adjoint");
    FNO_CUDA(sgemm(true, false, n, (int)mC, 2 * m, B, 1.f, f->Gi, n, 0, dHi, mC, sH, 1.f, f->Hx, 2 * mC, sX, s), "col adjoint");
    FNO_CUDA(sgemm(true, false, n, (int)mC, 2 * m, B, 1.f, f->Gr, n, 0, dHi, mC, sH, 0.f, f->Hx + mC, 2 * mC, sX, s), "col adjoint");
    FNO_CUDA(sgemm(true, false, n, (int)mC, 2 * m, B, -1.f, f->Gi, n, 0, dHr, mC, sH, 1.f, f->Hx + mC, 2 * mC, sX, s), "col adjoint");
    // dh_spec[q] = Fx^T dHx[q]
    if (f->tc_rows) {
      FNO_CUDA(run_xexpand(f, f->FxTB, f->Hx, (long long)B * n, f->dspec), "row adjoint (tensor cores)");
    } else {
      FNO_CUDA(sgemm(true, false, n, C, 2 * m, B * n, 1.f, f->Fx, n, 0, f->Hx, C, 2LL * m * C, 0.f, f->dspec, C,
                     (long long)n * C, s), "row adjoint");
    }
    // dh_l = dz W^T + dh_spec on the tensor cores
    PwArgs a;
    a.A = f->dzb;
    a.Bt = f->wbf + f->boff_Wn[l];
    a.bias = nullptr;
    a.add = f->dspec;
    a.out = f->dh;
    a.h = nullptr;
    a.hb = nullptr;
    a.P = P;
    a.err = f->tc_err;
    pointwise_tc_kernel<EPI_BWD><<<tc_grid(P), 128, 0, s>>>(a);
    FNO_CUDA(cudaGetLastError(), "pointwise adjoint");
  }
  // lift: dWp = x^T dh0, dbp = sum dh0
  return wgrad(f, x, f->cin, f->dh, C, P, f->grad + f->off_Wp, f->grad + f->off_bp);
}

}  // namespace

extern "C" {

ttsh_status ttsh_fno_create(const ttsh_fno_config* cfg, uint64_t seed, void* stream, ttsh_fno** out) {
  if (!out || !cfg) return fno_fail(TTSH_E_INVALID, "NULL argument");
  *out = nullptr;
  if (cfg->width != CW) return fno_fail(TTSH_E_UNSUPPORTED, "width must be 32");
  if (cfg->in_channels != 4) return fno_fail(TTSH_E_UNSUPPORTED, "in_channels must be 4");
  if (cfg->n < 16 || (cfg->n & (cfg->n - 1)) || cfg->n > 1024) return fno_fail(TTSH_E_INVALID, "n must be a power of two in [16, 1024]");
  if (cfg->modes < 1 || 2 * cfg->modes > cfg->n / 2) return fno_fail(TTSH_E_INVALID, "modes must be in [1, n/4]");
  if (cfg->layers < 1 || cfg->layers > 16 || cfg->max_batch < 1 || cfg->max_batch > 64)
    return fno_fail(TTSH_E_INVALID, "layers in [1, 16], max_batch in [1, 64]");
  ttsh_fno* f = new ttsh_fno();
  f->cfg = *cfg;
  f->stream = static_cast<cudaStream_t>(stream);
  f->n = cfg->n;
  f->C = cfg->width;
  f->m = cfg->modes;
  f->L = cfg->layers;
  f->cin = cfg->in_channels;
  f->Bmax = cfg->max_batch;
  f->nn = (long long)f->n * f->n;
  f->Pmax = f->nn * f->Bmax;
  const int C = f->C, m = f->m, L = f->L, n = f->n;
  const long long msz = 2LL * m * m * C * C;
  long long o = 0;
  f->off_Wp = o; o += (long long)f->cin * C;
  f->off_bp = o; o += C;
  for (int l = 0; l < L; ++l) {
    f->off_Wr.push_back(o); o += msz;
    f->off_Wi.push_back(o); o += msz;
    f->off_W.push_back(o); o += C * C;
    f->off_b.push_back(o); o += C;
  }
  f->off_Wq = o; o += C;
  f->off_bq = o; o += 1;
  f->nparams = o;
  long long bo = 0;
  for (int l = 0; l < L; ++l) {
    f->boff_Wr.push_back(bo); bo += msz;
    f->boff_Wi.push_back(bo); bo += msz;
    f->boff_Wt.push_back(bo); bo += C * C;
    f->boff_Wn.push_back(bo); bo += C * C;
  }
  auto cleanup = [&](ttsh_status st) {
    ttsh_fno_destroy(f);
    return st;
  };
  cudaError_t e = cudaSuccess;
  const long long P = f->Pmax, PC = P * C;
  const long long sH = 2LL * m * m * C;   // floats per sample of kept modes
  f->nwblk = 512;
  auto A = [&](auto** p, size_t bytes) {
    if (e == cudaSuccess) e = dalloc(f, p, bytes);
  };
  A(&f->theta, f->nparams * 4);
  A(&f->grad, f->nparams * 4);
  A(&f->adam_m, f->nparams * 4);
  A(&f->adam_v, f->nparams * 4);
  A(&f->wbf, bo * 2);
  A(&f->Fx, 2LL * m * n * 4);
  A(&f->Gr, 2LL * m * n * 4);
  A(&f->Gi, 2LL * m * n * 4);
  A(&f->Gpr, 2LL * m * n * 4);
  A(&f->Gpi, 2LL * m * n * 4);
  A(&f->Bx, 2LL * m * n * 4);
  A(&f->FxB, 32LL * n * 2);
  A(&f->BxB, 32LL * n * 2);
  A(&f->FxTB, 32LL * n * 2);
  A(&f->BxTB, 32LL * n * 2);
  f->h.assign(L + 1, nullptr);
  f->z.assign(L, nullptr);
  f->hb.assign(L, nullptr);
  f->Hr.assign(L, nullptr);
  f->Hi.assign(L, nullptr);
  for (int l = 0; l <= L; ++l) A(&f->h[l], PC * 4);
  for (int l = 0; l < L; ++l) {
    A(&f->z[l], PC * 4);
    A(&f->hb[l], PC * 2);
    A(&f->Hr[l], f->Bmax * sH * 4);
    A(&f->Hi[l], f->Bmax * sH * 4);
  }
  A(&f->Hx, (long long)f->Bmax * n * 2 * m * C * 4);
  A(&f->Yr, f->Bmax * sH * 4);
  A(&f->Yi, f->Bmax * sH * 4);
  A(&f->Z, (long long)f->Bmax * n * 2 * m * C * 4);
  A(&f->s, (PC > 2 * f->Bmax * sH ? PC : 2 * f->Bmax * sH) * 4);
  A(&f->dh, PC * 4);
  A(&f->dz, PC * 4);
  A(&f->dzb, PC * 2);
  A(&f->dspec, PC * 4);
  A(&f->dout, P * 4);
  A(&f->yo, P * 4);
  A(&f->wpart, (long long)f->nwblk * (C * C + C) * 4);
  A(&f->lpart, ((P + 255) / 256) * 8);
  A(&f->tc_err, 64);
  if (e == cudaSuccess) e = cudaMemsetAsync(f->tc_err, 0, 64, f->stream);
  if (e != cudaSuccess) return cleanup(fno_cuda(e, "FNO allocation"));
  // the fused column kernel needs its plan in shared memory
  if (column_fwd_mix_smem(n) <= 220 * 1024 && row_dft_smem(n, m) <= 220 * 1024 && 2 * m <= 64 &&
      (2 * m) % JB == 0 && n % YB == 0) {
    e = cudaFuncSetAttribute(column_fwd_mix_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             column_fwd_mix_smem(n));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(row_dft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, row_dft_smem(n, m));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(row_idft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, row_idft_smem(n, m));
    if (e != cudaSuccess) return cleanup(fno_cuda(e, "column kernel attribute"));
    f->fused_columns = true;
  }
  // DFT matrices on the kept modes
  {
    const double tp = 6.283185307179586476925286766559;
    std::vector<float> Fx(2 * m * n), Gr(2 * m * n), Gi(2 * m * n), Gpr(2 * m * n), Gpi(2 * m * n), Bx(2 * m * n);
    const double inv = 1.0 / ((double)n * n);
    for (int k = 0; k < m; ++k)
      for (int x = 0; x < n; ++x) {
        const double a = tp * (double)((long long)k * x % n) / n;
        Fx[k * n + x] = (float)cos(a);
        Fx[(m + k) * n + x] = (float)(-sin(a));
        const double c = k == 0 ? 1.0 : 2.0;
        Bx[x * 2 * m + k] = (float)(c * cos(a) * inv);
        Bx[x * 2 * m + m + k] = (float)(-c * sin(a) * inv);
      }
    for (int j = 0; j < 2 * m; ++j) {
      const int ky = j < m ? j : n - 2 * m + j;
      for (int y = 0; y < n; ++y) {
        const double a = tp * (double)((long long)ky * y % n) / n;
        Gr[j * n + y] = (float)cos(a);
        Gi[j * n + y] = (float)(-sin(a));
        Gpr[y * 2 * m + j] = (float)cos(a);
        Gpi[y * 2 * m + j] = (float)sin(a);
      }
    }
    const std::vector<float>* src[6] = {&Fx, &Gr, &Gi, &Gpr, &Gpi, &Bx};
    float* dst[6] = {f->Fx, f->Gr, f->Gi, f->Gpr, f->Gpi, f->Bx};
    for (int i = 0; i < 6 && e == cudaSuccess; ++i)
      e = cudaMemcpy(dst[i], src[i]->data(), src[i]->size() * 4, cudaMemcpyHostToDevice);
    // BF16 operands of the tensor-core row contractions, padded to 32 kept entries
    std::vector<__nv_bfloat16> fxb(32 * n), bxb(32 * n), fxtb(32 * n), bxtb(32 * n);
    for (int j = 0; j < 32; ++j)
      for (int x = 0; x < n; ++x) {
        const float fv = j < 2 * m ? Fx[j * n + x] : 0.f;
        const float bv = j < 2 * m ? Bx[x * 2 * m + j] : 0.f;
        fxb[j * n + x] = __float2bfloat16_rn(fv);    // [j][x]
        fxtb[x * 32 + j] = __float2bfloat16_rn(fv);  // [x][j]
        bxb[x * 32 + j] = __float2bfloat16_rn(bv);   // [x][j]
        bxtb[j * n + x] = __float2bfloat16_rn(bv);   // [j][x]
      }
    const std::vector<__nv_bfloat16>* bsrc[4] = {&fxb, &bxb, &fxtb, &bxtb};
    __nv_bfloat16* bdst[4] = {f->FxB, f->BxB, f->FxTB, f->BxTB};
    for (int i = 0; i < 4 && e == cudaSuccess; ++i)
      e = cudaMemcpy(bdst[i], bsrc[i]->data(), bsrc[i]->size() * 2, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cleanup(fno_cuda(e, "DFT matrices"));
    if (n % 16 == 0 && n <= kXcMaxN && 2 * m <= 32) {
      e = cudaFuncSetAttribute(xcontract_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, xcontract_smem(n));
      if (e != cudaSuccess) return cleanup(fno_cuda(e, "row contraction attribute"));
      f->tc_rows = true;
    }
  }
  // seeded initialisation: pointwise weights U(-1/sqrt(fan_in), 1/sqrt(fan_in)), biases 0,
  // spectral weights U(0, 1/(C*C)) (real and imaginary parts)
  {
    std::vector<float> th(f->nparams, 0.f);
    uint64_t ctr = 0;
    auto uni = [&](long long off, long long cnt, double lo, double hi) {
      for (long long i = 0; i < cnt; ++i) th[off + i] = (float)(lo + (hi - lo) * u01(seed, ctr++));
    };
    uni(f->off_Wp, (long long)f->cin * C, -1.0 / sqrt((double)f->cin), 1.0 / sqrt((double)f->cin));
    for (int l = 0; l < L; ++l) {
      uni(f->off_Wr[l], msz, 0.0, 1.0 / (C * C));
      uni(f->off_Wi[l], msz, 0.0, 1.0 / (C * C));
      uni(f->off_W[l], (long long)C * C, -1.0 / sqrt((double)C), 1.0 / sqrt((double)C));
    }
    uni(f->off_Wq, C, -1.0 / sqrt((double)C), 1.0 / sqrt((double)C));
    e = cudaMemcpy(f->theta, th.data(), th.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemsetAsync(f->adam_m, 0, f->nparams * 4, f->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(f->adam_v, 0, f->nparams * 4, f->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(f->grad, 0, f->nparams * 4, f->stream);
    if (e == cudaSuccess) e = refresh_bf16(f);
    if (e == cudaSuccess) e = cudaStreamSynchronize(f->stream);
    if (e != cudaSuccess) return cleanup(fno_cuda(e, "FNO initialisation"));
  }
  *out = f;
  return TTSH_OK;
}

void ttsh_fno_destroy(ttsh_fno* f) {
  if (!f) return;
  for (void* p : f->allocs) cudaFree(p);
  delete f;
}

int64_t ttsh_fno_num_params(const ttsh_fno* f) { return f ? f->nparams : -1; }

ttsh_status ttsh_fno_get_params(ttsh_fno* f, float* host) {
  if (!f || !host) return fno_fail(TTSH_E_INVALID, "NULL argument");
  FNO_CUDA(cudaMemcpyAsync(host, f->theta, f->nparams * 4, cudaMemcpyDeviceToHost, f->stream), "get params");
  FNO_CUDA(cudaStreamSynchronize(f->stream), "get params");
  return TTSH_OK;
}

ttsh_status ttsh_fno_set_params(ttsh_fno* f, const float* host) {
  if (!f || !host) return fno_fail(TTSH_E_INVALID, "NULL argument");
  FNO_CUDA(cudaMemcpyAsync(f->theta, host, f->nparams * 4, cudaMemcpyHostToDevice, f->stream), "set params");
  FNO_CUDA(refresh_bf16(f), "set params");
  FNO_CUDA(cudaStreamSynchronize(f->stream), "set params");
  return TTSH_OK;
}

ttsh_status ttsh_fno_set_scales(ttsh_fno* f, const float* in_scale, float out_scale) {
  if (!f || !in_scale || !(out_scale != 0.f)) return fno_fail(TTSH_E_INVALID, "bad scales");
  for (int i = 0; i < 4; ++i) f->in_scale[i] = in_scale[i];
  f->out_scale = out_scale;
  return TTSH_OK;
}

ttsh_status ttsh_fno_forward(ttsh_fno* f, const float* x, float* y, int32_t batch) {
  if (!f || !x || !y) return fno_fail(TTSH_E_INVALID, "NULL argument");
  if (batch < 1 || batch > f->Bmax) return fno_fail(TTSH_E_INVALID, "batch out of range");
  return forward_impl(f, x, batch, y, nullptr, nullptr);
}

ttsh_status ttsh_fno_loss_grad(ttsh_fno* f, const float* x, const float* target, int32_t batch, double* loss,
                               float* grad_host) {
  if (!f || !x || !target) return fno_fail(TTSH_E_INVALID, "NULL argument");
  if (batch < 1 || batch > f->Bmax) return fno_fail(TTSH_E_INVALID, "batch out of range");
  double l = 0;
  ttsh_status st = forward_impl(f, x, batch, f->yo, target, &l);
  if (st != TTSH_OK) return st;
  if ((st = backward_impl(f, x, batch, nullptr)) != TTSH_OK) return st;
  if (grad_host) {
    FNO_CUDA(cudaMemcpyAsync(grad_host, f->grad, f->nparams * 4, cudaMemcpyDeviceToHost, f->stream), "get grad");
  }
  FNO_CUDA(cudaStreamSynchronize(f->stream), "loss_grad");
  if ((st = check_tc(f)) != TTSH_OK) return st;
  if (loss) *loss = l;
  return TTSH_OK;
}

ttsh_status ttsh_fno_adam_step(ttsh_fno* f, float lr, float beta1, float beta2, float eps) {
  if (!f || !(lr > 0)) return fno_fail(TTSH_E_INVALID, "bad arguments");
  f->adam_t += 1;
  const float c1 = 1.f - powf(beta1, (float)f->adam_t), c2 = 1.f - powf(beta2, (float)f->adam_t);
  adam_kernel<<<(unsigned)((f->nparams + 255) / 256), 256, 0, f->stream>>>(f->theta, f->grad, f->adam_m, f->adam_v,
                                                                           f->nparams, lr, beta1, beta2, eps, c1, c2);
  FNO_CUDA(cudaGetLastError(), "adam");
  FNO_CUDA(refresh_bf16(f), "adam");
  return TTSH_OK;
}

ttsh_status ttsh_fno_features(ttsh_fno* f, ttsh_domain* d, float* x, int32_t sample) {
  if (!f || !d || !x) return fno_fail(TTSH_E_INVALID, "NULL argument");
  if (ttsh::domain_n(d) != f->n) return fno_fail(TTSH_E_INVALID, "domain grid differs from the network's");
  if (sample < 0 || sample >= f->Bmax) return fno_fail(TTSH_E_INVALID, "sample out of range");
  ttsh_status st = (ttsh_status)ttsh::domain_fields_to_staging(d);
  if (st != TTSH_OK) return st;
  cudaStream_t s = ttsh::domain_stream(d);
  const ttsh::DomainDev* dv = ttsh::domain_dev(d);
  float* xs = x + (long long)sample * f->nn * 4;
  const unsigned blk = (unsigned)((f->nn + 255) / 256);
  if (ttsh::domain_precision(d) == 32)
    features_kernel<float><<<blk, 256, 0, s>>>(dv->real, (const float*)dv->K, f->nn, f->in_scale[0], f->in_scale[1],
                                                f->in_scale[2], f->in_scale[3], xs);
  else
    features_kernel<double><<<blk, 256, 0, s>>>(dv->real, (const double*)dv->K, f->nn, f->in_scale[0],
                                                 f->in_scale[1], f->in_scale[2], f->in_scale[3], xs);
  FNO_CUDA(cudaGetLastError(), "features");
  return TTSH_OK;
}

ttsh_status ttsh_fno_rollout(ttsh_fno* f, ttsh_domain* d, int64_t nsteps, int32_t correct_every, float* scratch) {
  if (!f || !d || !scratch) return fno_fail(TTSH_E_INVALID, "NULL argument");
  if (nsteps < 0 || correct_every < 1 || correct_every > 64)
    return fno_fail(TTSH_E_INVALID, "nsteps >= 0 and correct_every in [1, 64] required");
  if (ttsh::domain_n(d) != f->n) return fno_fail(TTSH_E_INVALID, "domain grid differs from the network's");
  if (nsteps == 0) return TTSH_OK;
  // Record one period (correct_every solver steps + one correction) as a CUDA graph on a
  // private stream, then replay it on the domain's stream.
  cudaStream_t user = ttsh::domain_stream(d), cap = nullptr;
  FNO_CUDA(cudaStreamSynchronize(user), "rollout");
  FNO_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "rollout stream");
  const int64_t periods = nsteps / correct_every, rest = nsteps % correct_every;
  ttsh_status st = TTSH_OK;
  cudaGraphExec_t ge = nullptr;
  if (periods > 0) {
    // kernels must have their attributes set before capture: run one period eagerly
    if ((st = ttsh_step(d, correct_every)) == TTSH_OK) st = ttsh_fno_correct(f, d, scratch);
    if (st == TTSH_OK && periods > 1) {
      ttsh_set_stream(d, cap);
      cudaStream_t keep = f->stream;
      cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        st = ttsh_step(d, correct_every);
        if (st == TTSH_OK) st = ttsh_fno_correct(f, d, scratch);
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        if (st == TTSH_OK && e2 == cudaSuccess) e2 = cudaGraphInstantiate(&ge, g, 0);
        if (g) cudaGraphDestroy(g);
        if (st == TTSH_OK && e2 != cudaSuccess) st = fno_cuda(e2, "rollout capture");
      } else {
        st = fno_cuda(e, "rollout capture");
      }
      f->stream = keep;
      ttsh_set_stream(d, user);
      for (int64_t i = 1; i < periods && st == TTSH_OK; ++i) {
        cudaError_t e3 = cudaGraphLaunch(ge, user);
        if (e3 != cudaSuccess) st = fno_cuda(e3, "rollout replay");
      }
      // the capture counted one period that did not run; the replays ran periods - 1
      if (st == TTSH_OK) ttsh::domain_add_steps(d, (periods - 2) * (int64_t)correct_every);
    }
  }
  if (st == TTSH_OK && rest > 0) st = ttsh_step(d, rest);
  if (ge) cudaGraphExecDestroy(ge);
  cudaError_t e4 = cudaStreamSynchronize(user);
  cudaStreamDestroy(cap);
  if (st == TTSH_OK && e4 != cudaSuccess) st = fno_cuda(e4, "rollout");
  return st;
}

ttsh_status ttsh_fno_residual(ttsh_fno* f, ttsh_domain* truth, ttsh_domain* base, float* target, int32_t sample) {
  if (!f || !truth || !base || !target) return fno_fail(TTSH_E_INVALID, "NULL argument");
  if (ttsh::domain_n(truth) != f->n || ttsh::domain_n(base) != f->n)
    return fno_fail(TTSH_E_INVALID, "domain grid differs from the network's");
  if (sample < 0 || sample >= f->Bmax) return fno_fail(TTSH_E_INVALID, "sample out of range");
  ttsh_status st = (ttsh_status)ttsh::domain_fields_to_staging(truth);
  if (st != TTSH_OK) return st;
  st = (ttsh_status)ttsh::domain_fields_to_staging(base);
  if (st != TTSH_OK) return st;
  FNO_CUDA(cudaStreamSynchronize(ttsh::domain_stream(truth)), "residual");
  cudaStream_t s = ttsh::domain_stream(base);
  diff_kernel<<<(unsigned)((f->nn + 255) / 256), 256, 0, s>>>(ttsh::domain_dev(truth)->real,
                                                                ttsh::domain_dev(base)->real, f->nn, f->out_scale,
                                                                target + (long long)sample * f->nn);
  FNO_CUDA(cudaGetLastError(), "residual");
  FNO_CUDA(cudaStreamSynchronize(s), "residual");
  return TTSH_OK;
}

ttsh_status ttsh_fno_correct(ttsh_fno* f, ttsh_domain* d, float* scratch) {
  if (!f || !d || !scratch) return fno_fail(TTSH_E_INVALID, "NULL argument");
  ttsh_status st = ttsh_fno_features(f, d, scratch, 0);
  if (st != TTSH_OK) return st;
  float* y = scratch + f->nn * 4;
  cudaStream_t keep = f->stream;
  f->stream = ttsh::domain_stream(d);
  st = forward_impl(f, scratch, 1, y, nullptr, nullptr);
  f->stream = keep;
  if (st != TTSH_OK) return st;
  const ttsh::DomainDev* dv = ttsh::domain_dev(d);
  to_double_scaled_kernel<<<(unsigned)((f->nn + 255) / 256), 256, 0, ttsh::domain_stream(d)>>>(
      y, f->nn, 1.f / f->out_scale, dv->real);
  FNO_CUDA(cudaGetLastError(), "correction");
  return (ttsh_status)ttsh::domain_add_vorticity_from_staging(d);
}

}  // extern "C"
