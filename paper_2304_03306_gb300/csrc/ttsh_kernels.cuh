// ttsh_kernels.cuh - sm_103a kernels of the confined TTSH solver (templated on precision T
// and grid size N).
//
// One step of the integrating-factor Euler scheme of Appendix D (Algorithm 1) is two fused
// kernels:
//
//   row pass  (one block per R rows of the N x N box, real space)
//     inverse row transforms of omega^, v^x, v^y (column-transformed by the previous column
//     pass), giving omega, v_x, v_y in real space; then, per point,
//       F0 = c1 v_x + lambda v_y omega,  F1 = c1 v_y - lambda v_x omega,  F2 = -gamma_w K omega
//     with c1 = -b |v|^2 - gamma_v K, and forward row transforms of F0..F2, keeping only the
//     columns mx <= N/4 that the 1/2 rule can keep.
//
//   column pass (one block per stored column mx = 0..N/4, Fourier space)
//     forward column transforms of F0..F2; curl of the non-linear terms of Eq. (mod2),
//     rhs^ = i(kx F^1 - ky F^0) + F^2; integrating-factor Euler update
//     omega^ <- exp((a - (1 - k^2)^2) dt)(omega^ + dt rhs^); k = 0: omega^ = 0 and the mean
//     flow of Eq. (avg), v^(0) <- exp((a-1) dt)(v^(0) + dt R^1(0)) with R^1(0) = F^(0);
//     zero |m|^2 > (N/4)^2 (1/2 rule); Hermitian average (only the mx = 0 column needs it in
//     half-spectrum storage); then the stream function psi^ = omega^/k^2 and
//     v^ = (i ky psi^, -i kx psi^), and the inverse column transforms of omega^, v^x, v^y.
//
// Why this equals the non-linear terms of Eq. (mod2) as Appendix D writes them (velocity
// terms and v.grad(omega) in real space, then the curl): the advection term is taken in
// conservative form,
// v.grad(omega) = div(v omega), so i(kx F^1 - ky F^0) + F^2 = i(kx R^1y - ky R^1x)
// - lambda (i kx DFT[v_x omega] + i ky DFT[v_y omega]) - gamma_w DFT[K omega] = rhs^.  The two
// forms agree exactly (up to rounding) on every mode the update keeps: v and omega are
// band-limited to |m| <= N/4, so their grid product has no aliases inside that disc and its
// DFT there is the exact convolution, and k . v^(m) = 0 for every m (v comes from the stream
// function; k = 0 for the mean flow), so the convolution of i k omega^ with v^ equals
// i k times the convolution of omega^ with v^.  The k = 0 values are unchanged too:
// sum_x v omega = sum_m v^(m) conj(omega^(m)) = sum_m (i ky, -i kx) |omega^|^2 / k^2 = 0 (odd
// in m, and omega^(0) = 0).  This needs three inverse transforms per row and per column
// instead of five and four (no separate grad(omega) fields).
//
// Inter-pass buffers are column-major, [field][mx][y], so the column pass streams whole
// columns and the row pass reads/writes R consecutive y per column.  Every global input a
// block needs is first staged into shared memory with cp.async (all copies in flight at
// once, one wait), so the transform stages never wait on global memory.
#pragma once

#include <cuda.h>   // CUtensorMap (the tensor-map descriptor of the TMA loads)

#include "ttsh_fft.cuh"
#include "ttsh_wait.cuh"

namespace ttsh {

// ---------------------------------------------------------------------------------------
// Arguments (all device pointers belong to one domain's workspace)
// ---------------------------------------------------------------------------------------
// Write position and destination of the time series recorded by ttsh_step_record (set at the
// start of each call; the column pass of a recorded step appends one sample).
struct RecCtl {
  long long count;      // samples written in the current call
  long long base;       // step count of the first sample
  double* series;       // destination, 5 doubles per sample
  long long capacity;   // samples that fit
  double inv2n2;        // 1 / (2 N^2)
  int every;            // steps between samples
  int nblocks;          // row blocks whose partials make one sample
  int overflow;         // a sample did not fit (the host rejects such calls up front)
  int pad;
};

template <typename T>
struct Args {
  cplx<T>* what;        // state omega^, [mx][j], H x NK
  T* vmean;             // v^(0), 2 values
  T* K;                 // processed mask, N x N
  cplx<T>* G;           // column-pass output / row-pass input, [3][H][N]: omega, v_x, v_y
  cplx<T>* Rr;          // row-pass output / column-pass input, [3][H][N]
  const cplx<T>* tw;    // W_N^m, m in [0, N)
  double* real;         // double staging, [3][N][N]
  double* part;         // per-block diagnostic partial sums
  double* rec;          // per-block time-series partials of a recorded step, or null
  RecCtl* recctl;       // with rec: where the column pass appends the step's sample
  int* err;             // device status word: 1 = a bounded wait in a kernel ran out
  double* aux;          // two doubles: max |k.v^| and max |k||v^| of a divergence check
  int tma;              // 1: the row pass loads its G tile with the tensor-memory accelerator
  T a, b, lam, gv, gw, dt, dk, mean_decay;   // mean_decay = exp((a - 1) dt)
  double dx, cx, cy;    // grid spacing and the psi centre
};

enum RowKind { ROW_STEP = 0, ROW_FWD_VEL = 1, ROW_FWD_MASK = 2, ROW_INV_FIELDS = 3,
               ROW_INV_MASK = 4, ROW_INV_DIAG = 5 };
enum ColMode { COL_STEP = 0, COL_PROLOGUE = 1, COL_PROJECT = 2, COL_MASK = 3, COL_ADDW = 4, COL_DIV = 5 };

constexpr int kDiagQ = 5;   // per-block partials: sum|v|^2, sum w^2, sum|e_th.v|, sum|v|, #nonfinite
constexpr int kSmemLimit = 220 * 1024;
constexpr int kRecSmem = 32 * kDiagQ * 8 + 16;   // static shared memory: time-series reduction, TMA barrier

__host__ __device__ constexpr int align16(int v) { return (v + 15) / 16 * 16; }
__host__ __device__ constexpr int align128(int v) { return (v + 127) / 128 * 128; }

template <int KIND> __host__ __device__ constexpr int row_inv_fields() {
  return KIND == ROW_STEP ? 3 : KIND == ROW_INV_FIELDS ? 3 : KIND == ROW_INV_DIAG ? 3
       : KIND == ROW_INV_MASK ? 1 : 0;
}
// (the diagnostic pass also forward-transforms v_x, v_y for the divergence check)
template <int KIND> __host__ __device__ constexpr int row_fwd_fields() {
  return KIND == ROW_STEP ? 3 : KIND == ROW_FWD_VEL ? 2 : KIND == ROW_FWD_MASK ? 1 : KIND == ROW_INV_DIAG ? 2 : 0;
}

// Default tile shapes (the autotuner may pick others for the step kernels).
template <typename T, int N>
__host__ __device__ constexpr int default_rows() {
  return sizeof(T) == 4 ? (N <= 1024 ? 4 : N == 2048 ? 2 : 1) : (N <= 1024 ? 2 : 1);
}
template <typename T, int N>
__host__ __device__ constexpr int default_row_pe() { return sizeof(T) == 4 ? 16 : 8; }
template <typename T, int N>
__host__ __device__ constexpr int default_col_pe() { return sizeof(T) == 4 ? (N <= 1024 ? 8 : 16) : 8; }
// Tile shape of the step kernels' first variant (the plan a domain starts with).  As the
// defaults above, except the float 512^2 step, which starts with two rows per block and 16
// points per thread in both passes: the shape whose blocks are small enough (96 threads,
// < 45 KB of shared memory) for the persistent batched stepper to keep several resident per
// SM; the autotuner may pick the faster single-domain shape.  (At 256^2 and 128^2 two rows
// and 8 points per thread are faster for one domain alone - 3.3 against 4.2 us, 2.6 against
// 3.7 us per row pass - but slower in a batch, where twice the blocks pay their fixed costs
// twice: 53.0 against 49.9 us per step of the 48-domain sweep; so they stay autotuner
// choices.)
template <typename T, int N>
__host__ __device__ constexpr int default_step_rows() { return sizeof(T) == 4 && N == 512 ? 2 : default_rows<T, N>(); }
template <typename T, int N>
__host__ __device__ constexpr int default_step_row_pe() { return default_row_pe<T, N>(); }
template <typename T, int N>
__host__ __device__ constexpr int default_step_col_pe() { return sizeof(T) == 4 && N == 512 ? 16 : default_col_pe<T, N>(); }
// blocks per cluster of the default step row pass (8192^2 float: one row per block, pairs)
template <typename T, int N>
__host__ __device__ constexpr int default_row_cluster() { return sizeof(T) == 4 && N >= 8192 ? 2 : 1; }

// Stride between the row buffers of one block: R-strided accesses (prep writes, post reads)
// land on distinct banks when consecutive rows are 32/R banks apart.
__host__ __device__ constexpr int row_stride(int LP, int R, int words) {
  return R == 1 ? LP : LP + ((((32 / R) / words) % (32 / words) - LP % (32 / words)) % (32 / words) + (32 / words)) % (32 / words);
}

// Blocks of a kernel with `smem` bytes of dynamic shared memory that fit an SM's 228 KB,
// counting the 1 KB the runtime reserves per block and up to kRecSmem of static shared memory.
__host__ __device__ constexpr int smem_blocks_per_sm(int smem) { return (228 * 1024) / (smem + kRecSmem + 1024); }

// Row-pass geometry and shared-memory plan.  CL > 1: the step kernel runs as clusters of CL
// blocks over CL * R consecutive rows; each block stages one CL-th of the stored columns for
// all the cluster's rows (global segments of CL * R values instead of R), and the blocks
// read from each other's shares through distributed shared memory.  CMP = 1 (compact): the
// forward transforms work in place (no separate buffers) and the mask rows are read from
// global memory where the real-space terms need them (not staged), so that two or more
// blocks fit per SM on large grids and one block's staging and stores overlap another's
// transforms.
template <typename T, int N, int KIND, int R, int PEV, int CL = 1, int CMP = 0>
struct RowGeo {
  static constexpr int L = N / 2, M = N / 4, H = M + 1;
  static constexpr int PE = cmin(PEV, L);
  static constexpr int PS = pad_shift<T>();
  static constexpr int LP = padded_len<L, PS>();
  static constexpr int TT = L / PE;
  static constexpr int FI = row_inv_fields<KIND>();
  static constexpr int FF = row_fwd_fields<KIND>();
  static constexpr int F = cmax(FI, FF);
  static constexpr int NPL = FI;   // G planes read (field f comes from plane f)
  static constexpr int CB = (int)sizeof(cplx<T>);
  static constexpr int LPR = row_stride(LP, R, CB / 4);
  static constexpr int TW_BYTES = align16(TwTab<T, N>::ENTRIES * CB) + StageTab<T, L, PE>::BYTES;
  static constexpr int OFF_STAB = align16(TwTab<T, N>::ENTRIES * CB);
  // every region starts on a 16-byte boundary (16-byte cp.async destinations)
  static constexpr int BUF_BYTES = align16(F * R * LPR * CB);
  // staged G tile: plane f at OFF_GIN + f * GPS ([mx][r] inside a plane); planes start on
  // 128-byte boundaries, as tensor-memory-accelerator destinations must.  With clusters a
  // block stages HC columns (its share) of RS rows (the cluster's).
  static constexpr int HC = (H + CL - 1) / CL;
  static constexpr int RS = R * CL;
  static constexpr int GIN_DENSE = NPL * align128(HC * RS * CB);   // decides what is staged
  static constexpr int KS_BYTES = KIND == ROW_STEP ? align16(R * N * (int)sizeof(T)) : 0;
  static constexpr int RED_BYTES = KIND == ROW_INV_DIAG ? kDiagQ * 1024 * 8 : 0;
  static constexpr bool STAGE_K = KS_BYTES > 0 && CMP == 0 && TW_BYTES + BUF_BYTES + KS_BYTES + RED_BYTES <= kSmemLimit;
  static constexpr bool STAGE_G = GIN_DENSE > 0 &&
      TW_BYTES + BUF_BYTES + GIN_DENSE + (STAGE_K ? KS_BYTES : 0) + RED_BYTES <= kSmemLimit;
  // step kernel: the forward transforms get buffers of their own when they fit, so that the
  // real-space terms can be the first forward stage's input functor (read from the inverse
  // buffers, no in-place pass)
  // (float only: in double the duplicated c1 arithmetic costs more DP-pipe time than the
  // saved pass)
  static constexpr bool SEPARATE = KIND == ROW_STEP && sizeof(T) == 4 && STAGE_K && CMP == 0 &&
      TW_BYTES + 2 * BUF_BYTES + (STAGE_G ? GIN_DENSE : 0) + KS_BYTES <= kSmemLimit;
  // Slots per mx in a staged plane.  The first inverse stage reads one row's consecutive mx
  // across the lanes of a half-warp (8-byte values) or quarter-warp (16-byte values): with an
  // odd number of slots per mx they meet every bank once; with an even one (R slots) two or
  // four of them share a bank.  So without clusters (whose shares are exchanged in 16-byte
  // pieces) an even R gets one spare slot, where the padded tile still fits the budget that
  // decided the staging above.
  // Nor may the padding cost a block per SM (batched launches run several per SM): the
  // padded plan must leave as many blocks per SM as the dense one.
  static constexpr int RS_ODD = RS % 2 == 1 ? RS : RS + 1;
  static constexpr int PAD_EXTRA = STAGE_G ? NPL * (align128(HC * RS_ODD * CB) - align128(HC * RS * CB)) : 0;
  static constexpr int SMEM_DENSE = align128(TW_BYTES + BUF_BYTES) + (STAGE_G ? GIN_DENSE : 0) +
      (STAGE_K ? KS_BYTES : 0) + RED_BYTES + (SEPARATE ? BUF_BYTES : 0) + 128;
  static constexpr bool PAD_G = CL == 1 && STAGE_G && RS_ODD != RS &&
      TW_BYTES + (SEPARATE ? 2 : 1) * BUF_BYTES + GIN_DENSE + PAD_EXTRA + (STAGE_K ? KS_BYTES : 0) + RED_BYTES <=
          kSmemLimit &&
      smem_blocks_per_sm(SMEM_DENSE + PAD_EXTRA) == smem_blocks_per_sm(SMEM_DENSE);
  static constexpr int RSP = PAD_G ? RS_ODD : RS;
  static constexpr int GPS = align128(HC * RSP * CB);
  static constexpr int GIN_BYTES = NPL * GPS;
  static constexpr int OFF_BUF = TW_BYTES;
  static constexpr int OFF_GIN = align128(OFF_BUF + BUF_BYTES);
  static constexpr int OFF_KS = OFF_GIN + (STAGE_G ? GIN_BYTES : 0);
  static constexpr int OFF_RED = OFF_KS + (STAGE_K ? KS_BYTES : 0);
  static constexpr int OFF_FWD = OFF_RED + RED_BYTES;
  // + 128: the kernel aligns its dynamic shared-memory base to 128 bytes
  static constexpr int SMEM = OFF_FWD + (SEPARATE ? BUF_BYTES : 0) + 128;
  static_assert(SMEM == SMEM_DENSE + (PAD_G ? PAD_EXTRA : 0), "shared-memory plan and its dense estimate disagree");
  // the G tile can come by TMA: one box of R rows x (N/4+1) columns per plane (at most 256
  // columns in a box; a row segment of R complex values a multiple of 16 bytes)
  static constexpr bool TMA_OK = CL == 1 && STAGE_G && !PAD_G && H <= 256 && (R * CB) % 16 == 0;
  static constexpr int NT = cmax(64, cmin(1024, F * R * TT));
  static constexpr int SEG = RS * CB;                       // bytes per (plane, mx) segment
  static constexpr int SEGP = RSP * CB;                     // bytes between consecutive segments
  static constexpr int CHUNK = SEG % 16 == 0 && SEGP % 16 == 0 ? 16 : 8;
  static constexpr bool VALID = SMEM + (KIND == ROW_STEP ? kRecSmem : 0) <= 227 * 1024 && N % R == 0 &&
                                R <= N && TT <= 1024 && NT % TT == 0 &&
                                (CL == 1 || (CL == 2 && KIND == ROW_STEP && STAGE_G && (N / R) % CL == 0 &&
                                             SEG % 16 == 0));
  static_assert(OFF_BUF % 16 == 0 && OFF_GIN % 128 == 0 && GPS % 128 == 0 && OFF_KS % 16 == 0 &&
                OFF_RED % 16 == 0 && OFF_FWD % 16 == 0,
                "row pass shared-memory regions must be 16-byte (G tile: 128-byte) aligned");
};

// Column-pass geometry and shared-memory plan.
template <typename T, int N, int MODE, int PEV>
struct ColGeo {
  static constexpr int M = N / 4, H = M + 1, NK = 2 * M + 1;
  static constexpr int PE = cmin(PEV, N);
  static constexpr int PS = pad_shift<T>();
  static constexpr int LP = padded_len<N, PS>();
  static constexpr int TT = N / PE;
  static constexpr int NF = MODE == COL_STEP ? 3 : (MODE == COL_PROJECT || MODE == COL_DIV) ? 2
                         : (MODE == COL_MASK || MODE == COL_ADDW) ? 1 : 0;
  static constexpr int NI = MODE == COL_MASK ? 1 : MODE == COL_DIV ? 0 : 3;
  static constexpr int CB = (int)sizeof(cplx<T>);
  static constexpr int TW_BYTES = align16(TwTab<T, N>::ENTRIES * CB) + StageTab<T, N, PE>::BYTES;
  static constexpr int OFF_STAB = align16(TwTab<T, N>::ENTRIES * CB);
  static constexpr int ACC_BYTES = align16(NK * CB);
  static constexpr int WS_BYTES = (MODE == COL_STEP || MODE == COL_ADDW || MODE == COL_DIV) ? align16(NK * CB) : 0;
  static constexpr int FIXED = TW_BYTES + ACC_BYTES + WS_BYTES + 64;
  static constexpr int FB0 = cmax(NF, NI) >= 4 ? 4 : cmax(NF, NI);
  static constexpr int FB = (FIXED + FB0 * LP * CB <= kSmemLimit) ? FB0
                          : (FIXED + 2 * LP * CB <= kSmemLimit && FB0 >= 2) ? 2 : 1;
  // forward inputs in one batch: the NF columns can come as bulk copies (contiguous in Rr)
  // into an unpadded staging area that the first transform stage reads
  static constexpr int STG_BYTES = NF * N * CB;
  static constexpr bool BULK = NF > 0 && FB >= NF && FIXED + FB * LP * CB + STG_BYTES <= kSmemLimit;
  static constexpr int OFF_BUF = TW_BYTES;
  static constexpr int OFF_ACC = OFF_BUF + align16(FB * LP * CB);
  static constexpr int OFF_WS = OFF_ACC + ACC_BYTES;
  static constexpr int OFF_STG = OFF_WS + WS_BYTES;
  static constexpr int OFF_S0 = OFF_STG + (BULK ? STG_BYTES : 0);
  static constexpr int SMEM = OFF_S0 + 64;
  // transforms in flight at once: as many of the FB as fit in the thread budget; with 16
  // points per thread the budget is 768 threads (85 registers each), since 1024 threads
  // (64 registers) make the radix-16 butterflies spill
  static constexpr int NTCAP = PE >= 16 ? 768 : 1024;
  static constexpr int NT = cmax(64, TT * cmax(1, cmin(FB, NTCAP / TT)));
  static constexpr bool VALID = SMEM <= 227 * 1024 && TT <= 1024 && NT % TT == 0 && NT <= 1024;
  static_assert(OFF_BUF % 16 == 0 && OFF_ACC % 16 == 0 && OFF_WS % 16 == 0 && OFF_STG % 16 == 0 &&
                OFF_S0 % 16 == 0,
                "column pass shared-memory regions must be 16-byte aligned");
};

// ---------------------------------------------------------------------------------------
// Time-series sample taken inside a step's row pass.  The pass already holds omega, v_x and
// v_y of its R rows in real space (the state the step starts from), so the energy,
// enstrophy and order-parameter sums cost one sweep over shared memory spread over all the
// block's threads (in the in-place variants, the loop of the real-space terms, which reads
// every point once anyway): per-thread, per-warp and per-block sums in T (fixed order), one
// partial per block written to A.rec; the column pass's sample block adds the partials up.
// Same quantities as ROW_INV_DIAG: sum |v|^2, sum omega^2, sum |e_theta . v| (e_theta = 0 at
// the centre), sum |v|, number of points with a non-finite value.
// ---------------------------------------------------------------------------------------
template <typename T>
struct SeriesSums {
  T s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  int bad = 0;
  // point (x, y) of the grid with omega = w, v = (vx, vy); (px, py) its position relative
  // to the centre
  __device__ __forceinline__ void add(T w, T vx, T vy, T px, T py) {
    const T rr2 = px * px + py * py;
    const T v2 = vx * vx + vy * vy;
    s0 += v2;
    s1 += w * w;
    s2 += rr2 > (T)0 ? fabs(px * vy - py * vx) * rsqrt(rr2) : (T)0;
    if constexpr (sizeof(T) == 4) s3 += v2 > (T)0 ? v2 * rsqrt(v2) : (T)0;   // |v| within 2 ulp
    else s3 += sqrt(v2);
    bad += (isfinite(w) && isfinite(vx) && isfinite(vy)) ? 0 : 1;
  }
  // every thread of the NT calls this once: warp sums in T (fixed-order shuffles), then the
  // warps in index order, also in T (one barrier), to the block's partial blk of A.rec
  // (kDiagQ values of type T).  No double arithmetic here (on GB300 a double add costs the
  // SM's FP64 unit 16 cycles per warp): the column pass's sample block adds the block
  // partials up.
  template <int NT>
  __device__ __forceinline__ void store(const Args<T>& A, int blk) const {
    T q[kDiagQ] = {s0, s1, s2, s3, (T)bad};   // per-thread counts are small: exact in T
    constexpr int NW = (NT + 31) / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wl = cmin(32, NT - warp * 32);   // lanes present in this warp
    const unsigned mask = wl == 32 ? 0xffffffffu : ((1u << wl) - 1u);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
      for (int k = 0; k < kDiagQ; ++k) {
        const T o = __shfl_down_sync(mask, q[k], off);
        if (lane + off < wl) q[k] += o;
      }
    }
    __shared__ T wsum[NW][kDiagQ];
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < kDiagQ; ++k) wsum[warp][k] = q[k];
    }
    block_sync<NT>();
    if (threadIdx.x < kDiagQ) {
      T t = wsum[0][threadIdx.x];
#pragma unroll
      for (int w2 = 1; w2 < NW; ++w2) t += wsum[w2][threadIdx.x];
      reinterpret_cast<T*>(A.rec)[(size_t)blk * kDiagQ + threadIdx.x] = t;
    }
  }
};

// Double-float sums (value = hi + lo, |lo| <= ulp(hi) / 2): Knuth's error-free TwoSum, so
// adding up float partials this way is as accurate as adding them in double, at the float
// rate (on GB300 one double add costs the SM's FP64 unit 16 cycles per warp).
struct DFloat {
  float hi, lo;   // trivial, so that it can live in shared memory; start from {0, 0}
  __device__ __forceinline__ static void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
  }
  __device__ __forceinline__ void add(float x) {
    float s, e;
    two_sum(hi, x, s, e);
    hi = s;
    lo += e;
  }
  __device__ __forceinline__ void add(DFloat o) {
    float s, e;
    two_sum(hi, o.hi, s, e);
    e += lo + o.lo;
    hi = s + e;                 // renormalise (|e| small against s)
    lo = e - (hi - s);
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Append {step, energy, enstrophy, psi, non-finite count} from the five sums.
__device__ __forceinline__ void record_append(RecCtl* c, const double* t) {
  const double two_over_pi = 0.63661977236758134307553505349005744813783858296183;
  const long long i = c->count;
  if (i < c->capacity) {
    double* o = c->series + (size_t)i * 5;
    o[0] = (double)(c->base + i * (long long)c->every);
    o[1] = t[0] * c->inv2n2;
    o[2] = t[1] * c->inv2n2;
    o[3] = (t[2] / t[3] - two_over_pi) / (1.0 - two_over_pi);
    o[4] = t[4];
  } else {
    c->overflow = 1;
  }
  c->count = i + 1;
}

// Finish a recorded step's sample (one extra block of the column pass, which runs beside the
// column blocks): warp 0 adds the row pass's block partials up in a fixed order (lane l
// takes partials l, l + 32, ...; then a shuffle tree), as double-float sums for a float
// domain and in double for a double one, and appends {step, energy, enstrophy, psi,
// non-finite count}.  The other warps leave at once: on the path to the next step, one
// warp's short dependent chain costs less than a cross-warp reduction.
template <typename T>
__device__ __forceinline__ void record_sample(const Args<T>& A) {
  griddep_launch();
  griddep_wait();   // the row pass's partials
  if (threadIdx.x >= 32) return;   // the block has at least 64 threads: warp 0 is whole
  RecCtl* c = A.recctl;
  const T* part = reinterpret_cast<const T*>(A.rec);
  const int lane = threadIdx.x;
  const int np = c->nblocks;
  using Acc = typename std::conditional<sizeof(T) == 4, DFloat, double>::type;
  Acc q[kDiagQ];
#pragma unroll
  for (int k = 0; k < kDiagQ; ++k) q[k] = Acc{};   // zero: {0, 0} or 0.0
  for (int b = lane; b < np; b += 32)
#pragma unroll
    for (int k = 0; k < kDiagQ; ++k) {
      if constexpr (sizeof(T) == 4) q[k].add(part[(size_t)b * kDiagQ + k]);
      else q[k] += part[(size_t)b * kDiagQ + k];
    }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
#pragma unroll
    for (int k = 0; k < kDiagQ; ++k) {
      if constexpr (sizeof(T) == 4) {
        DFloat o;
        o.hi = __shfl_down_sync(0xffffffffu, q[k].hi, off);
        o.lo = __shfl_down_sync(0xffffffffu, q[k].lo, off);
        q[k].add(o);
      } else {
        q[k] += __shfl_down_sync(0xffffffffu, q[k], off);
      }
    }
  if (lane == 0) {
    double r[kDiagQ];
#pragma unroll
    for (int k = 0; k < kDiagQ; ++k) {
      if constexpr (sizeof(T) == 4) r[k] = q[k].value();
      else r[k] = q[k];
    }
    record_append(c, r);
  }
}

// ---------------------------------------------------------------------------------------
// Thread-block clusters: rank, barrier, distributed shared memory
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// Every thread of every block of the cluster arrives; shared-memory writes before it are
// visible to every block of the cluster after it (a hardware barrier, no polling).
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
// Address of the same shared-memory location in block `rank` of this cluster.
__device__ __forceinline__ unsigned dsmem_addr(const void* p, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
               : "=r"(r) : "r"((unsigned)__cvta_generic_to_shared(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ cplx<float> dsmem_ld(unsigned a, float) {
  float x, y;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(x), "=f"(y) : "r"(a) : "memory");
  return mk<float>(x, y);
}
__device__ __forceinline__ cplx<double> dsmem_ld(unsigned a, double) {
  double x, y;
  asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(x), "=d"(y) : "r"(a) : "memory");
  return mk<double>(x, y);
}
__device__ __forceinline__ void dsmem_st(unsigned a, cplx<float> v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void dsmem_st(unsigned a, cplx<double> v) {
  asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(a), "d"(v.x), "d"(v.y) : "memory");
}

// ---------------------------------------------------------------------------------------
// Row pass body (one block = rows [y0, y0 + R))
// ---------------------------------------------------------------------------------------
// With CL = 2 (clusters of two blocks over 2R consecutive rows) block c of a cluster stages
// the stored columns [c HC, c HC + HC) of both blocks' rows (global segments of 2R values),
// slot (j, s) of a plane holding column c HC + j of the cluster's row s (s < R: block 0's
// rows, s >= R: block 1's).  The first inverse stage reads the other block's share through
// distributed shared memory; the forward results go back the same way into the share that
// owns their column, and each block writes its share for all 2R rows.  Three cluster
// barriers: shares staged; every block past its inverse loads (the shares are then
// overwritten); results in place.
// tmapG: G as a 2D tensor [3 (N/4+1)][2N scalars] with a box of R rows x (N/4+1), a grid-
// constant kernel parameter (used when A.tma is set; may be null otherwise).
// REC = false leaves out the time-series sums (for callers whose Args never carry them).
template <typename T, int N, int KIND, int R, int PEV, int CL = 1, int CMP = 0, bool REC = true>
__device__ __forceinline__ void row_body(const Args<T>& A, int blk, unsigned char* smem_raw,
                                         const CUtensorMap* tmapG) {
  using Geo = RowGeo<T, N, KIND, R, PEV, CL, CMP>;
  static_assert(Geo::VALID, "row pass tile does not fit");
  constexpr int L = Geo::L, M = Geo::M, H = Geo::H;
  constexpr int NT = Geo::NT, PE = Geo::PE, PS = Geo::PS, LP = Geo::LPR;
  constexpr int FI = Geo::FI, FF = Geo::FF;
  cplx<T>* sm = reinterpret_cast<cplx<T>*>(smem_raw + Geo::OFF_BUF);
  cplx<T>* gin = reinterpret_cast<cplx<T>*>(smem_raw + Geo::OFF_GIN);
  T* ks = reinterpret_cast<T*>(smem_raw + Geo::OFF_KS);
  const int y0 = blk * R;
  const int tid = threadIdx.x;
  constexpr int GPC = Geo::GPS / Geo::CB;   // G-tile plane stride in complex values
  const int crank = CL > 1 ? (int)cluster_rank() : 0;
  const int yc = y0 - crank * R;            // first row of the cluster
  const int cbase = crank * Geo::HC;        // first stored column of this block's share
  const int ccnt = cmin(Geo::HC, H - cbase);

  // ---- stage: twiddles and the K rows (inputs no previous kernel writes), then, once the
  // previous kernel has finished, the G tile (R consecutive y of every stored column) ----
  const TwTab<T, N> tw = TwTab<T, N>::fill(reinterpret_cast<cplx<T>*>(smem_raw), A.tw, tid, NT);
  cplx<T>* stab = reinterpret_cast<cplx<T>*>(smem_raw + Geo::OFF_STAB);
  StageTab<T, L, PE>::template fill<N>(stab, A.tw, tid, NT);
  if constexpr (Geo::STAGE_K) {
    constexpr int NCH = R * N * (int)sizeof(T) / 16;
    const char* src = reinterpret_cast<const char*>(A.K + (size_t)y0 * N);
    for (int i = tid; i < NCH; i += NT) cp_async16(reinterpret_cast<char*>(ks) + 16 * i, src + 16 * i);
  }
  griddep_wait();
  if constexpr (Geo::STAGE_G) {
    bool via_tma = false;
    if constexpr (Geo::TMA_OK) via_tma = A.tma != 0 && tmapG != nullptr;
    if (via_tma) {
      // one tensor-memory-accelerator load per plane: box (R consecutive y) x (all N/4+1
      // columns) of G, landing as [mx][r]; completion counted in bytes on an mbarrier
      __shared__ __align__(8) unsigned long long tma_bar;
      const unsigned bar = (unsigned)__cvta_generic_to_shared(&tma_bar);
      if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      }
      block_sync<NT>();
      if (tid == 0) {
        constexpr unsigned bytes = (unsigned)(Geo::NPL * H * R * Geo::CB);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
        for (int pl = 0; pl < Geo::NPL; ++pl) {
          const unsigned dst = (unsigned)__cvta_generic_to_shared(reinterpret_cast<char*>(gin) + pl * Geo::GPS);
          const int x = 2 * y0, y = pl * H;   // scalar column (16-byte aligned: R * CB % 16 == 0), row
          asm volatile(
              "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
              ::"r"(dst), "l"(tmapG), "r"(x), "r"(y), "r"(bar) : "memory");
        }
      }
      if (!mbar_wait_bounded(bar, 0, kWaitLimitNs)) atomicExch(A.err, 1);
    } else {
      constexpr int CPS = Geo::SEG / Geo::CHUNK;   // chunks per (plane, mx) segment
#pragma unroll
      for (int pl = 0; pl < Geo::NPL; ++pl) {
        const char* gsrc = reinterpret_cast<const char*>(A.G + ((size_t)pl * H + cbase) * N + yc);
        char* gdst = reinterpret_cast<char*>(gin) + pl * Geo::GPS;
        for (int i = tid; i < ccnt * CPS; i += NT)   // i = j * CPS + c: the plane is [mx][r]
          cp_async<Geo::CHUNK>(gdst + (i / CPS) * Geo::SEGP + (i % CPS) * Geo::CHUNK,
                               gsrc + (size_t)(i / CPS) * N * Geo::CB + (i % CPS) * Geo::CHUNK);
      }
    }
  }
  cp_async_wait_all();   // tables and staged inputs
  block_sync<NT>();

  if constexpr (CL > 1) cluster_sync();   // every block's share is staged and visible

  // ---- inverse row transforms (C2R through an L-point complex transform) ----
  // The twiddle pre-pass that turns the half spectrum X of a real row into the L-point
  // complex input Z[k] = (X[k] + conj X[L-k]) + i conj(W_N^k) (X[k] - conj X[L-k]) is the
  // input functor of the first transform stage.
  if constexpr (FI > 0) {
    auto load = [&](int bt, int k) -> cplx<T> {
      const int f = bt / R, r = bt % R;   // field f (omega, v_x, v_y / the mask) from G plane f
      cplx<T> X = mk<T>(0, 0), Xm = mk<T>(0, 0);
      const int km = L - k;
      if constexpr (Geo::STAGE_G) {
        if constexpr (CL == 1) {
          const cplx<T>* src = gin + (size_t)f * GPC + r;
          if (k <= M) X = src[k * Geo::RSP];
          if (km <= M) Xm = src[km * Geo::RSP];
        } else {
          // column kk of this block's row r: slot (kk - o HC, c R + r) of the share of block
          // o that owns it, read through distributed shared memory when o is the other block
          auto get = [&](int kk) -> cplx<T> {
            const int o = kk < Geo::HC ? 0 : 1;
            const int idx = f * GPC + (kk - o * Geo::HC) * Geo::RS + crank * R + r;
            return o == crank ? gin[idx] : dsmem_ld(dsmem_addr(gin + idx, (unsigned)o), T());
          };
          if (k <= M) X = get(k);
          if (km <= M) Xm = get(km);
        }
      } else {
        const cplx<T>* src = A.G + (size_t)f * H * N + (y0 + r);
        if (k <= M) X = src[(size_t)k * N];
        if (km <= M) Xm = src[(size_t)km * N];
      }
      if (k == 0) X.y = 0;   // the mx = 0 entry of a real row is real
      const cplx<T> w = conjg(tw.get(k));        // conj(W_N^k)
      const cplx<T> s = X + conjg(Xm);
      const cplx<T> d = X - conjg(Xm);
      return s + mul_i(cmul(w, d));
    };
    fft_batch<T, L, PE, +1, NT, N, LP>(sm, FI * R, tw, stab, load);
  }

  // ---- real-space work ----
  // element x of a real row lives in complex slot x/2 (re for even x, im for odd x)
  auto rl = [&](int f, int r, int x) -> T& {
    cplx<T>& c = sm[(f * R + r) * LP + padi<PS>(x >> 1)];
    return (x & 1) ? c.y : c.x;
  };

  cplx<T>* fw = sm;   // buffers of the forward transforms
  if constexpr (KIND == ROW_INV_DIAG) fw = sm + R * LP;   // v_x, v_y (fields 1 and 2)
  if constexpr (KIND == ROW_STEP && Geo::SEPARATE) {
    fw = reinterpret_cast<cplx<T>*>(smem_raw + Geo::OFF_FWD);
    // F0..F2 at complex slot k of row r (real points 2k in .x, 2k + 1 in .y), computed from
    // omega, v_x, v_y and K as the forward transforms' input; same arithmetic as the
    // in-place loop below
    auto rhs = [&](int bt, int k) -> cplx<T> {
      const int f = bt / R, r = bt % R;
      const cplx<T> wz = sm[(0 * R + r) * LP + padi<PS>(k)];
      // the slot's two mask values in one load (the staged rows start 16-byte aligned, N is even)
      const cplx<T> kk = reinterpret_cast<const cplx<T>*>(ks + r * N)[k];
      const T k0 = kk.x, k1 = kk.y;
      if (f == 2) return mk<T>(-(A.gw * k0) * wz.x, -(A.gw * k1) * wz.y);
      const cplx<T> vxz = sm[(1 * R + r) * LP + padi<PS>(k)];
      const cplx<T> vyz = sm[(2 * R + r) * LP + padi<PS>(k)];
      auto F = [&](T w, T vx, T vy, T Kv) -> T {
        const T v2 = fma(vx, vx, vy * vy);
        const T c1 = fma(-A.b, v2, -(A.gv * Kv));
        const T lw = A.lam * w;
        return f == 0 ? fma(c1, vx, lw * vy) : fma(c1, vy, -(lw * vx));
      };
      return mk<T>(F(wz.x, vxz.x, vyz.x, k0), F(wz.y, vxz.y, vyz.y, k1));
    };
    if (REC && A.rec != nullptr) {
      // a recorded step: one sweep over the real-space fields, spread over every thread of
      // the block, adds each point to the time-series sums (the fields stay in place: the
      // forward transforms write a separate buffer)
      SeriesSums<T> ss;
      const T dx = (T)A.dx, cx = (T)A.cx, cy = (T)A.cy;
#pragma unroll 4
      for (int e = tid; e < R * N; e += NT) {
        const int r = e / N, x = e % N;
        ss.add(rl(0, r, x), rl(1, r, x), rl(2, r, x), (T)(x - N / 2) * dx - cx, (T)(y0 + r - N / 2) * dx - cy);
      }
      ss.template store<NT>(A, blk);
    }
    fft_batch<T, L, PE, -1, NT, N, LP>(fw, FF * R, tw, stab, rhs);
  } else if constexpr (KIND == ROW_STEP) {
    // the real-space terms in place; a recorded step also adds every point to the
    // time-series sums as it reads it
    auto terms = [&](auto rec_tag) {
      constexpr bool RS = decltype(rec_tag)::value;
      SeriesSums<T> ss;
      const T dx = (T)A.dx, cx = (T)A.cx, cy = (T)A.cy;
      for (int e = tid; e < R * N; e += NT) {
        const int r = e / N, x = e % N;
        const T w = rl(0, r, x), vx = rl(1, r, x), vy = rl(2, r, x);
        if constexpr (RS) ss.add(w, vx, vy, (T)(x - N / 2) * dx - cx, (T)(y0 + r - N / 2) * dx - cy);
        T Kv;
        if constexpr (Geo::STAGE_K) Kv = ks[e];
        else Kv = A.K[(size_t)(y0 + r) * N + x];
        // explicit fused multiply-adds: every kernel instantiation (single and batched)
        // rounds the same way
        const T v2 = fma(vx, vx, vy * vy);
        const T c1 = fma(-A.b, v2, -(A.gv * Kv));        // velocity terms: -b|v|^2 v - gamma_v K v = c1 v
        const T lw = A.lam * w;                           // advection, conservative form
        rl(0, r, x) = fma(c1, vx, lw * vy);
        rl(1, r, x) = fma(c1, vy, -(lw * vx));
        rl(2, r, x) = -(A.gw * Kv) * w;
      }
      if constexpr (RS) ss.template store<NT>(A, blk);
    };
    if (REC && A.rec != nullptr) terms(std::true_type{});
    else terms(std::false_type{});
  } else if constexpr (KIND == ROW_FWD_VEL || KIND == ROW_FWD_MASK) {
    for (int e = tid; e < FF * R * N; e += NT) {
      const int x = e % N;
      const int t = e / N;
      const int r = t % R, f = t / R;
      rl(f, r, x) = (T)A.real[((size_t)f * N + (y0 + r)) * N + x];
    }
  } else if constexpr (KIND == ROW_INV_FIELDS) {
    for (int e = tid; e < 3 * R * N; e += NT) {
      const int x = e % N;
      const int t = e / N;
      const int r = t % R, f = t / R;
      A.real[((size_t)f * N + (y0 + r)) * N + x] = (double)rl(f, r, x);
    }
  } else if constexpr (KIND == ROW_INV_MASK) {
    for (int e = tid; e < R * N; e += NT) {
      const int r = e / N, x = e % N;
      const T k = rl(0, r, x);
      A.K[(size_t)(y0 + r) * N + x] = k * k;          // K = (iDFT[...])^2
    }
  } else if constexpr (KIND == ROW_INV_DIAG) {
    double acc[kDiagQ] = {0, 0, 0, 0, 0};
    for (int e = tid; e < R * N; e += NT) {
      const int r = e / N, x = e % N;
      const double w = (double)rl(0, r, x);
      const double vx = (double)rl(1, r, x), vy = (double)rl(2, r, x);
      const double px = (x - N / 2) * A.dx - A.cx;
      const double py = (y0 + r - N / 2) * A.dx - A.cy;
      const double rr = sqrt(px * px + py * py);
      const double vn = sqrt(vx * vx + vy * vy);
      acc[0] += vx * vx + vy * vy;
      acc[1] += w * w;
      acc[2] += rr > 0 ? fabs(-py * vx + px * vy) / rr : 0.0;
      acc[3] += vn;
      acc[4] += (isfinite(w) && isfinite(vx) && isfinite(vy)) ? 0.0 : 1.0;
    }
    // fixed-order block reduction (deterministic)
    double* red = reinterpret_cast<double*>(smem_raw + Geo::OFF_RED);
    for (int q = 0; q < kDiagQ; ++q) red[q * 1024 + tid] = acc[q];
    block_sync<NT>();
    for (int s = 512; s >= 1; s >>= 1) {
      if (tid < s && tid + s < NT)
        for (int q = 0; q < kDiagQ; ++q) red[q * 1024 + tid] += red[q * 1024 + tid + s];
      block_sync<NT>();
    }
    if (tid < kDiagQ) A.part[(size_t)blk * kDiagQ + tid] = red[tid * 1024];
  }

  // ---- forward row transforms (R2C), keep mx <= N/4 ----
  if constexpr (FF > 0) {
    if constexpr (!Geo::SEPARATE) fft_batch<T, L, PE, -1, NT, N, LP>(fw, FF * R, tw, stab);
    // programmatic dependent launch: the next pass may be launched now that this block only
    // has its stores left (triggering earlier lets the next pass's waiting blocks take shared
    // memory from this pass's blocks that have not started yet)
    griddep_launch();
    // clusters: every block is past its inverse loads, so the shares can take the results
    if constexpr (CL > 1) cluster_sync();
    for (int e = tid; e < FF * R * H; e += NT) {
      const int r = e % R;
      const int t = e / R;
      const int k = t % H;
      const int f = t / H;
      const cplx<T>* row = fw + (f * R + r) * LP;
      const cplx<T> Zk = row[padi<PS>(k)];
      const cplx<T> Zm = conjg(row[padi<PS>((L - k) & (L - 1))]);
      const cplx<T> s = Zk + Zm;
      const cplx<T> d = Zk - Zm;
      // X[k] = (Zk + Zm)/2 - (i/2) W^k (Zk - Zm)
      const cplx<T> X = (s - mul_i(cmul(tw.get(k), d))) * (T)0.5;
      if constexpr (CL == 1) {
        A.Rr[((size_t)f * H + k) * N + (y0 + r)] = X;
      } else {
        // into slot (column, this block's row) of the share that owns column k
        const int o = k < Geo::HC ? 0 : 1;
        const int idx = f * GPC + (k - o * Geo::HC) * Geo::RS + crank * R + r;
        if (o == crank) gin[idx] = X;
        else dsmem_st(dsmem_addr(gin + idx, (unsigned)o), X);
      }
    }
    if constexpr (CL > 1) {
      cluster_sync();   // every row's results of this block's share are in place
      // write the share: per plane and column, the cluster's RS consecutive y in 16-byte pieces
      constexpr int PPS = Geo::SEG / 16;
      for (int i = tid; i < FF * ccnt * PPS; i += NT) {
        const int f = i / (ccnt * PPS), rem = i - f * (ccnt * PPS);
        const int j = rem / PPS, pz = rem - j * PPS;
        const uint4 v = *reinterpret_cast<const uint4*>(reinterpret_cast<const char*>(gin) + f * Geo::GPS +
                                                        j * Geo::SEG + pz * 16);
        *reinterpret_cast<uint4*>(reinterpret_cast<char*>(A.Rr + ((size_t)f * H + cbase + j) * N + yc) + pz * 16) = v;
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// Column pass body (one block = stored column mx = kx)
// ---------------------------------------------------------------------------------------
template <typename T, int N, int MODE, int PEV>
__device__ __forceinline__ void col_body(const Args<T>& A, int kx, unsigned char* smem_raw) {
  using Geo = ColGeo<T, N, MODE, PEV>;
  static_assert(Geo::VALID, "column pass tile does not fit");
  constexpr int M = Geo::M, H = Geo::H, NK = Geo::NK;
  constexpr int PE = Geo::PE, PS = Geo::PS, LP = Geo::LP, NT = Geo::NT, FB = Geo::FB;
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw + Geo::OFF_BUF);
  cplx<T>* acc = reinterpret_cast<cplx<T>*>(smem_raw + Geo::OFF_ACC);
  cplx<T>* ws = reinterpret_cast<cplx<T>*>(smem_raw + Geo::OFF_WS);
  T* s0 = reinterpret_cast<T*>(smem_raw + Geo::OFF_S0);   // [0..1]: k = 0 forward values, [2..3]: v^(0)
  const int tid = threadIdx.x;
  const T kxp = A.dk * (T)kx;
  const T invN = (T)1 / (T)N;
  constexpr int CB = Geo::CB;

  const TwTab<T, N> tw = TwTab<T, N>::fill(reinterpret_cast<cplx<T>*>(smem_raw), A.tw, tid, NT);
  cplx<T>* stab = reinterpret_cast<cplx<T>*>(smem_raw + Geo::OFF_STAB);
  StageTab<T, N, PE>::template fill<N>(stab, A.tw, tid, NT);
  griddep_wait();   // everything below reads what the previous kernel wrote
  auto ky_of = [](int j) { return j <= M ? j : j - NK; };
  // async copy of nb contiguous columns of Rr (fields f0..f0+nb-1) into the padded buffers
  auto stage_columns = [&](int f0, int nb) {
    for (int e = tid; e < nb * N; e += NT) {
      const int b = e / N, y = e % N;
      cp_async<CB>(buf + b * LP + padi<PS>(y), A.Rr + ((size_t)(f0 + b) * H + kx) * N + y);
    }
  };

  // ---- forward column transforms and curl assembly ----
  if constexpr (MODE != COL_PROLOGUE) {
    constexpr int NF = Geo::NF;
    if constexpr (MODE == COL_STEP || MODE == COL_ADDW) {
      for (int j = tid; j < NK; j += NT) cp_async<CB>(ws + j, A.what + (size_t)kx * NK + j);
    }
    if constexpr (Geo::BULK) {
      // the NF columns (each N contiguous values of Rr) by bulk copies, completion counted
      // in bytes on an mbarrier (bounded wait)
      __shared__ __align__(8) unsigned long long col_bar;
      const unsigned bar = (unsigned)__cvta_generic_to_shared(&col_bar);
      if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      }
      block_sync<NT>();
      if (tid == 0) {
        constexpr unsigned bytes = (unsigned)(NF * N * CB);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
        for (int f = 0; f < NF; ++f) {
          const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_raw + Geo::OFF_STG + (size_t)f * N * CB);
          asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                       ::"r"(dst), "l"(A.Rr + ((size_t)f * H + kx) * N), "r"((unsigned)(N * CB)), "r"(bar)
                       : "memory");
        }
      }
      if (!mbar_wait_bounded(bar, 0, kWaitLimitNs) && A.err) atomicExch(A.err, 1);
    }
    for (int f0 = 0; f0 < NF; f0 += FB) {
      const int nb = cmin(FB, NF - f0);
      if constexpr (Geo::BULK) {
        const cplx<T>* stg = reinterpret_cast<const cplx<T>*>(smem_raw + Geo::OFF_STG);
        cp_async_wait_all();   // tables, state column
        fft_batch<T, N, PE, -1, NT, N>(buf, nb, tw, stab, [&](int bt, int m) { return stg[bt * N + m]; });
      } else {
        stage_columns(f0, nb);
        cp_async_wait_all();
        fft_batch<T, N, PE, -1, NT, N>(buf, nb, tw, stab);
      }
      for (int j = tid; j < NK; j += NT) {
        const int ky = ky_of(j);
        const int idx = ky & (N - 1);
        const T kyp = A.dk * (T)ky;
        cplx<T> a = f0 == 0 ? mk<T>(0, 0) : acc[j];
        T q2 = (T)0;   // COL_DIV: |v^x|^2 + |v^y|^2
        if constexpr (MODE == COL_DIV) q2 = f0 == 0 ? (T)0 : ws[j].x;
        for (int b = 0; b < nb; ++b) {
          const int f = f0 + b;
          const cplx<T> v = buf[b * LP + padi<PS>(idx)];
          if constexpr (MODE == COL_MASK || MODE == COL_ADDW) {
            a = v;
          } else if constexpr (MODE == COL_DIV) {
            // f = 0: v^x -> kx; f = 1: v^y -> ky (k . v^)
            a = a + v * (f == 0 ? kxp : kyp);
            q2 += v.x * v.x + v.y * v.y;
          } else {
            // f = 0: (F0 | v_x) -> -i ky; f = 1: (F1 | v_y) -> +i kx; f = 2: F2 -> 1
            if (f == 0) a = a - mul_i(v) * kyp;
            else if (f == 1) a = a + mul_i(v) * kxp;
            else a = a + v;
            if (kx == 0 && j == 0 && f < 2) s0[f] = v.x;   // raw k = 0 value (real)
          }
        }
        acc[j] = a;
        if constexpr (MODE == COL_DIV) ws[j].x = q2;
      }
      block_sync<NT>();   // buf is refilled by the next batch
    }

    if constexpr (MODE == COL_DIV) {
      // largest |k.v^| and |k||v^| over the stored modes of the 1/2-rule disc, in double;
      // maxima of non-negative doubles combine as their bit patterns (order-independent)
      double dmax = 0.0, kvmax = 0.0;
      for (int j = tid; j < NK; j += NT) {
        const int ky = ky_of(j);
        const int m2 = kx * kx + ky * ky;
        if (m2 > M * M) continue;
        const double ax = (double)acc[j].x, ay = (double)acc[j].y;
        const double dkd = (double)A.dk;
        dmax = fmax(dmax, sqrt(ax * ax + ay * ay));
        kvmax = fmax(kvmax, dkd * sqrt((double)m2) * sqrt((double)ws[j].x));
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        dmax = fmax(dmax, __shfl_down_sync(0xffffffffu, dmax, off));
        kvmax = fmax(kvmax, __shfl_down_sync(0xffffffffu, kvmax, off));
      }
      if ((tid & 31) == 0) {
        atomicMax(reinterpret_cast<unsigned long long*>(A.aux), (unsigned long long)__double_as_longlong(dmax));
        atomicMax(reinterpret_cast<unsigned long long*>(A.aux) + 1, (unsigned long long)__double_as_longlong(kvmax));
      }
    }

    if constexpr (MODE != COL_DIV) {   // the divergence check ends with its maxima
      // ---- update: integrating-factor Euler, k = 0, 1/2 rule ----
      for (int j = tid; j < NK; j += NT) {
        const int ky = ky_of(j);
        const int m2 = kx * kx + ky * ky;
        cplx<T> wn;
        if constexpr (MODE == COL_STEP) {
          const T k2 = A.dk * A.dk * (T)m2;
          const T om = (T)1 - k2;
          const T E = exp((A.a - om * om) * A.dt);
          const cplx<T> w = ws[j];
          const cplx<T> r = acc[j] * invN;
          wn = (w + r * A.dt) * E;
          if (m2 == 0 || m2 > M * M) wn = mk<T>(0, 0);
        } else if constexpr (MODE == COL_PROJECT) {
          wn = acc[j] * invN;
          if (m2 == 0 || m2 > M * M) wn = mk<T>(0, 0);
        } else if constexpr (MODE == COL_ADDW) {
          // correction delta^ = DFT[delta omega] on the 1/2-rule disc, delta^(0) = 0
          wn = acc[j] * invN;
          if (m2 == 0 || m2 > M * M) wn = mk<T>(0, 0);
        } else {   // COL_MASK: keep |m|^2 <= (N/8)^2, fold both 1/N factors of the round trip
          wn = acc[j] * (invN * invN);
          if (m2 > (N / 8) * (N / 8)) wn = mk<T>(0, 0);
        }
        acc[j] = wn;
      }
      if constexpr (MODE == COL_STEP || MODE == COL_PROJECT) {
        if (kx == 0 && tid == 0) {
          for (int c = 0; c < 2; ++c) {
            T vm;
            if constexpr (MODE == COL_STEP)
              vm = A.mean_decay * (A.vmean[c] + A.dt * (s0[c] * invN));   // Eq. (avg)
            else
              vm = s0[c] * invN;                                              // DFT[v](0)
            s0[2 + c] = vm;
            A.vmean[c] = vm;
          }
        }
      }
      block_sync<NT>();
      if constexpr (MODE == COL_STEP || MODE == COL_PROJECT || MODE == COL_ADDW) {
        // Hermitian average; with half-spectrum storage only mx = 0 pairs are stored
        if (kx == 0) {
          for (int ky = 1 + tid; ky <= M; ky += NT) {
            const cplx<T> p = acc[ky], q = acc[NK - ky];
            const cplx<T> h = (p + conjg(q)) * (T)0.5;
            acc[ky] = h;
            acc[NK - ky] = conjg(h);
          }
          block_sync<NT>();
        }
        if constexpr (MODE == COL_ADDW) {
          for (int j = tid; j < NK; j += NT) acc[j] = acc[j] + ws[j];
          if (kx == 0 && tid == 0) {
            s0[2] = A.vmean[0];
            s0[3] = A.vmean[1];
          }
          block_sync<NT>();
        }
        for (int j = tid; j < NK; j += NT) A.what[(size_t)kx * NK + j] = acc[j];
      }
    }
  } else {
    for (int j = tid; j < NK; j += NT) acc[j] = A.what[(size_t)kx * NK + j];
    if (kx == 0 && tid == 0) {
      s0[2] = A.vmean[0];
      s0[3] = A.vmean[1];
    }
    cp_async_wait_all();   // tables
    block_sync<NT>();
  }

  if constexpr (MODE != COL_DIV) {
    // ---- inverse column transforms of the fields the next row pass reads ----
    constexpr int NI = Geo::NI;
    for (int f0 = 0; f0 < NI; f0 += FB) {
      const int nb = cmin(FB, NI - f0);
      // spectral multipliers of the four fields, applied as the first stage's input functor
      auto load = [&](int bt, int idx) -> cplx<T> {
        const int f = f0 + bt;
        const int ky = idx <= N / 2 ? idx : idx - N;
        cplx<T> v = mk<T>(0, 0);
        if (ky >= -M && ky <= M) {
          const cplx<T> w = acc[ky >= 0 ? ky : ky + NK];
          if constexpr (MODE == COL_MASK) {
            v = w;
          } else {
            const T kyp = A.dk * (T)ky;
            const int m2 = kx * kx + ky * ky;
            const T k2 = A.dk * A.dk * (T)m2;
            const T inv = m2 > 0 ? invN / k2 : (T)0;
            if (f == 0) v = w * invN;                       // omega
            else if (f == 1) v = mul_i(w) * (kyp * inv);    // v^x = i ky psi^   (stream function)
            else v = mul_i(w) * (-kxp * inv);               // v^y = -i kx psi^
            if (m2 == 0 && f >= 1) v = mk<T>(s0[2 + (f - 1)] * invN, (T)0);   // mean flow
          }
        }
        return v;
      };
      fft_batch<T, N, PE, +1, NT, N, 0>(buf, nb, tw, stab, load);
      if (f0 + nb >= NI) griddep_launch();   // only the last stores are left (see the row pass)
      for (int e = tid; e < nb * N; e += NT) {
        const int b = e / N, y = e % N;
        A.G[((size_t)(f0 + b) * H + kx) * N + y] = buf[b * LP + padi<PS>(y)];
      }
      block_sync<NT>();
    }
  }
}

// ---------------------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------------------
// Dynamic shared memory re-based to a 128-byte boundary (TMA destinations need it; the row
// geometry reserves the slack).
__device__ __forceinline__ unsigned char* smem_base128(unsigned char* raw) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(raw);
  return raw + ((128u - (a & 127u)) & 127u);
}

// The tensor map is a separate grid-constant parameter so that its address can be handed to
// the TMA while the argument block stays an ordinary by-value parameter.
template <typename T, int N, int KIND, int R, int PEV, int CL = 1, int CMP = 0>
__global__ void __launch_bounds__(RowGeo<T, N, KIND, R, PEV, CL, CMP>::NT)
row_kernel(Args<T> A, const __grid_constant__ CUtensorMap tmapG) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  row_body<T, N, KIND, R, PEV, CL, CMP>(A, blockIdx.x, smem_base128(smem_raw), &tmapG);
}

template <typename T, int N, int MODE, int PEV>
__global__ void __launch_bounds__(ColGeo<T, N, MODE, PEV>::NT)
col_kernel(Args<T> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if constexpr (MODE == COL_STEP) {
    if (blockIdx.x == ColGeo<T, N, MODE, PEV>::H) {   // launched only for a recorded step
      static_assert(ColGeo<T, N, MODE, PEV>::NT >= 32, "the sample block needs a whole warp 0");
      record_sample(A);
      return;
    }
  }
  col_body<T, N, MODE, PEV>(A, blockIdx.x, smem_raw);
}

// Batched variants: blockIdx.y selects the domain, whose arguments live in a device array.
template <typename T, int N, int KIND, int R, int PEV>
__global__ void __launch_bounds__(RowGeo<T, N, KIND, R, PEV>::NT)
row_kernel_batched(const Args<T>* __restrict__ args) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Args<T> A = args[blockIdx.y];   // tma is 0 and rec null in packed argument blocks
  row_body<T, N, KIND, R, PEV, 1, 0, false>(A, blockIdx.x, smem_base128(smem_raw), nullptr);
}

template <typename T, int N, int MODE, int PEV>
__global__ void __launch_bounds__(ColGeo<T, N, MODE, PEV>::NT)
col_kernel_batched(const Args<T>* __restrict__ args) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Args<T> A = args[blockIdx.y];
  col_body<T, N, MODE, PEV>(A, blockIdx.x, smem_raw);
}

// ---------------------------------------------------------------------------------------
// Diagnostics reductions (fixed order, double precision)
// ---------------------------------------------------------------------------------------
// Sum nblocks x kDiagQ partials into out[kDiagQ] with one block of 256 threads.
__global__ void diag_reduce_kernel(const double* __restrict__ part, int nblocks, double* out);

// Per-column shell spectrum: one thread per (stored column kx, shell s).  Shell s holds the
// modes with round(|m|) = s, i.e. s^2 - s + 1 <= m^2 <= s^2 + s (s >= 1; s = 0: m = 0), so in
// column kx its modes are two contiguous ranges of ky (ky >= 0 and ky < 0); each thread sums
// them in the storage order of the column.  The s = 0 thread of each column also counts the
// column's non-finite values.
__device__ __forceinline__ int isqrt_floor(long long v) {
  if (v <= 0) return 0;
  long long r = (long long)sqrt((double)v);
  while (r * r > v) --r;
  while ((r + 1) * (r + 1) <= v) ++r;
  return (int)r;
}

template <typename T, int N>
__global__ void spectrum_col_kernel(Args<T> A, int nbins, double* __restrict__ colhist,
                                    int* __restrict__ badcount) {
  constexpr int M = N / 4, NK = 2 * M + 1;
  const int kx = blockIdx.y;
  const int sh = blockIdx.x * blockDim.x + threadIdx.x;
  if (sh >= nbins) return;
  const cplx<T>* col = A.what + (size_t)kx * NK;
  const double dk = (double)A.dk;
  const double wgt = kx > 0 ? 2.0 : 1.0;   // mx > 0 columns stand for +-mx
  auto energy = [&](int ky) {
    const int m2 = kx * kx + ky * ky;
    if (m2 == 0) {
      const double u = (double)A.vmean[0], v = (double)A.vmean[1];
      return u * u + v * v;
    }
    const cplx<T> w = col[ky >= 0 ? ky : ky + NK];
    const double wr = (double)w.x, wi = (double)w.y;
    return (wr * wr + wi * wi) / (dk * dk * (double)m2);
  };
  double h = 0.0;
  const long long s2 = (long long)sh * sh;
  const long long lo2 = sh == 0 ? 0 : s2 - sh + 1, hi2 = sh == 0 ? 0 : s2 + sh;   // range of m^2
  const long long k2 = (long long)kx * kx;
  if (hi2 >= k2) {
    const int ylo = lo2 - k2 <= 0 ? 0 : isqrt_floor(lo2 - k2 - 1) + 1;   // smallest ky >= 0 with ky^2 >= lo2 - kx^2
    const int yhi = isqrt_floor(hi2 - k2 < 0 ? 0 : hi2 - k2);
    const int top = yhi < M ? yhi : M;
    for (int ky = ylo; ky <= top; ++ky) h += wgt * energy(ky);
    const int nlo = ylo > 1 ? ylo : 1;
    for (int ky = -top; ky <= -nlo; ++ky) h += wgt * energy(ky);
  }
  colhist[(size_t)kx * nbins + sh] = h;
  if (sh == 0) {
    int bad = 0;
    for (int j = 0; j < NK; ++j)
      if (!isfinite((double)col[j].x) || !isfinite((double)col[j].y)) ++bad;
    if (bad) atomicAdd(badcount, bad);
  }
}

__global__ void spectrum_reduce_kernel(const double* __restrict__ colhist, int ncols, int nbins,
                                       double scale, double* __restrict__ out);

}  // namespace ttsh
