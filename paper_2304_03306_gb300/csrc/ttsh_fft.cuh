// ttsh_fft.cuh - shared-memory FFT building blocks for the sm_103a solver kernels.
//
// The solver's transforms are the unitary DFT pair of Appendix D, applied separably: real
// row transforms (length N, done as N/2-point complex transforms plus a twiddle pass) and
// complex column transforms (length N).  Everything here is un-normalised; the kernels
// apply the 1/N factors where the update needs them.
//
// Transform engine: in-place Stockham autosort with radix-PE register butterflies.  Each
// transform of length L is owned by L/PE threads; in every stage a thread loads PE values
// (PE/R butterflies of radix R), all threads synchronise, each applies the inter-stage
// twiddles, an R-point DFT in registers (radix-2 decimation in frequency, output in
// bit-reversed register order) and writes the results to their Stockham positions.  Shared
// memory is padded by one slot every 128 bytes (16 float or 8 double complex values),
// whatever PE is: the stages' 8- and 16-byte accesses are served 128 bytes per wavefront,
// and with this interval the contiguous runs a thread writes in the first stage, and the
// strided reads of the later stages, fall on distinct banks (one slot every PE elements did
// the same only for PE = 16 in float and PE = 8 in double).
//
// Twiddles W_N^m = exp(-2 pi i m / N) come from shared memory (the whole table when it fits
// in 16 KB, else two tables of ~sqrt(N) entries whose product gives W_N^m; per-stage tables
// when they fit in 32 KB), copied asynchronously once per block from a correctly rounded
// global table together with the block's other inputs; no stage waits on global memory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace ttsh {

// Aligned to its size, so that a complex value moves as one 8- or 16-byte access (every
// buffer holding them - shared-memory regions, the workspace - is 16-byte aligned).
template <typename T>
struct alignas(2 * sizeof(T)) cplx {
  T x, y;
};

template <typename T>
__device__ __forceinline__ cplx<T> mk(T x, T y) {
  cplx<T> r;
  r.x = x;
  r.y = y;
  return r;
}
template <typename T>
__device__ __forceinline__ cplx<T> operator+(cplx<T> a, cplx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T>
__device__ __forceinline__ cplx<T> operator-(cplx<T> a, cplx<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename T>
__device__ __forceinline__ cplx<T> operator*(cplx<T> a, T s) { return mk(a.x * s, a.y * s); }
template <typename T>
__device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T>
__device__ __forceinline__ cplx<T> conjg(cplx<T> a) { return mk(a.x, -a.y); }
// i * a
template <typename T>
__device__ __forceinline__ cplx<T> mul_i(cplx<T> a) { return mk(-a.y, a.x); }

__host__ __device__ constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v >> 1); }
__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }

// Padded shared-memory index: one spare slot every 2^PS elements.
template <typename T>
__host__ __device__ constexpr int pad_shift() { return ilog2(128 / (int)sizeof(cplx<T>)); }
template <int PS>
__device__ __forceinline__ int padi(int i) { return i + (i >> PS); }
template <int L, int PS>
__host__ __device__ constexpr int padded_len() { return L + (L >> PS); }

template <int R>
__device__ __forceinline__ constexpr int bitrev(int i) {
  int r = 0;
  for (int b = 1; b < R; b <<= 1) {
    r = (r << 1) | (i & 1);
    i >>= 1;
  }
  return r;
}

// cos(2 pi j / 16) for j = 0..4 (exact decimal expansions of cos 0, cos pi/8, cos pi/4,
// cos 3pi/8, cos pi/2); other angles follow by symmetry.
__device__ __forceinline__ constexpr double cos16(int j) {
  return j == 0 ? 1.0
       : j == 1 ? 0.92387953251128675612818318939678828682241662586364
       : j == 2 ? 0.70710678118654752440084436210484903928483593768847
       : j == 3 ? 0.38268343236508977172845998403039886676134456248563
       : 0.0;
}

// d * exp(DIR * 2 pi i j / 16), j in [0, 8), DIR = -1 (forward) or +1 (inverse).
template <typename T, int DIR>
__device__ __forceinline__ cplx<T> rot16(cplx<T> d, int j) {
  if (j == 0) return d;
  if (j == 4) return DIR > 0 ? mul_i(d) : mk(d.y, -d.x);
  const T c = (T)(j <= 4 ? cos16(j) : -cos16(8 - j));
  const T s = (T)(DIR) * (T)(j <= 4 ? cos16(4 - j) : cos16(j - 4));
  return mk(d.x * c - d.y * s, d.x * s + d.y * c);
}

// In-register R-point DFT (R <= 16), sign DIR.  Radix-2 decimation in frequency: on exit
// v[bitrev(k)] holds X[k].
template <typename T, int R, int DIR>
__device__ __forceinline__ void dft_reg(cplx<T>* v) {
#pragma unroll
  for (int half = R / 2; half >= 1; half >>= 1) {
#pragma unroll
    for (int blk = 0; blk < R; blk += 2 * half) {
#pragma unroll
      for (int i = 0; i < half; ++i) {
        const cplx<T> a = v[blk + i];
        const cplx<T> b = v[blk + i + half];
        v[blk + i] = a + b;
        v[blk + i + half] = rot16<T, DIR>(a - b, i * (16 / (2 * half)));
      }
    }
  }
}

// Asynchronous global -> shared copies (cp.async, completion tracked per thread).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
// Programmatic dependent launch: let the next kernel in the stream start its prologue, and
// wait until the previous kernel has completed and its writes are visible.  Both are no-ops
// for a kernel launched without the programmatic-serialization attribute.
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  if constexpr (BYTES == 16) cp_async16(smem, gmem);
  else if constexpr (BYTES == 8) cp_async8(smem, gmem);
  else cp_async4(smem, gmem);
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_all;\n" ::: "memory");
}

// Twiddle table in shared memory for W_TWN^m, m in [0, TWN): the full table when it takes at
// most 16 KB, otherwise two levels W^m = W^{(m >> S) 2^S} * W^{m mod 2^S}.
template <typename T, int TWN>
struct TwTab {
  static constexpr bool FULL = TWN * (int)sizeof(cplx<T>) <= 16384;
  static constexpr int LOG = ilog2(TWN);
  static constexpr int SB = FULL ? LOG : (LOG + 1) / 2;
  static constexpr int NLO = 1 << SB;
  static constexpr int NHI = TWN >> SB;
  static constexpr int ENTRIES = NLO + NHI;
  const cplx<T>* lo;   // W^i,          i < NLO
  const cplx<T>* hi;   // W^(i * NLO),  i < NHI
  __device__ __forceinline__ cplx<T> get(int m) const {
    if constexpr (NHI == 1) {
      return lo[m];
    } else {
      return cmul(hi[m >> SB], lo[m & (NLO - 1)]);
    }
  }
  // Fill from the global table with cp.async (all threads of the block); the caller waits
  // (cp_async_wait_all) and synchronises before the first use.
  __device__ __forceinline__ static TwTab fill(cplx<T>* sm, const cplx<T>* __restrict__ tw, int tid, int nt) {
    for (int i = tid; i < ENTRIES; i += nt)
      cp_async<(int)sizeof(cplx<T>)>(sm + i, i < NLO ? tw + i : tw + (size_t)(i - NLO) * NLO);
    TwTab t;
    t.lo = sm;
    t.hi = sm + NLO;
    return t;
  }
};

template <typename T, int DIR, typename TW>
__device__ __forceinline__ cplx<T> twiddle(const TW& tw, int idx) {
  cplx<T> w = tw.get(idx);
  if (DIR > 0) w.y = -w.y;
  return w;
}

// Per-stage twiddle tables.  Stage (Ns, R) of a length-L transform multiplies input r of the
// butterfly with sub-index k by W_TWN^{r k TWN/(Ns R)}; stored as [r - 1][k] (k fastest) those
// reads are contiguous across a warp, where indexing one W_TWN table with stride r*k would
// put many threads on the same bank.  Used when all stages' tables fit in 32 KB.
__host__ __device__ constexpr int stage_radix(int L, int PE, int Ns) { return (L / Ns < PE) ? L / Ns : PE; }
__host__ __device__ constexpr int stage_offset(int L, int PE, int NsTarget) {
  int off = 0;
  for (int Ns = 1; Ns < NsTarget; Ns *= stage_radix(L, PE, Ns))
    if (Ns > 1) off += (stage_radix(L, PE, Ns) - 1) * Ns;
  return off;
}

template <typename T, int L, int PE>
struct StageTab {
  static constexpr int ENTRIES = stage_offset(L, PE, L);
  static constexpr bool USE = ENTRIES > 0 && ENTRIES * (int)sizeof(cplx<T>) <= 32768;
  static constexpr int BYTES = USE ? (ENTRIES * (int)sizeof(cplx<T>) + 15) / 16 * 16 : 0;
  // fill from the global W_TWN table with cp.async (all threads; the caller waits and
  // synchronises before the first use)
  template <int TWN>
  __device__ __forceinline__ static void fill(cplx<T>* sm, const cplx<T>* __restrict__ tw, int tid, int nt) {
    if constexpr (USE) {
      int off = 0;
      for (int Ns = 1; Ns < L; Ns *= stage_radix(L, PE, Ns)) {
        const int R = stage_radix(L, PE, Ns);
        if (Ns > 1) {
          const int stride = TWN / (Ns * R);
          for (int i = tid; i < (R - 1) * Ns; i += nt) {
            const int r = 1 + i / Ns, k = i % Ns;
            cp_async<(int)sizeof(cplx<T>)>(sm + off + i, tw + (size_t)r * k * stride);
          }
          off += (R - 1) * Ns;
        }
      }
    }
  }
};

// Block barrier over the NT threads that run a pass body: a named hardware barrier (id 1)
// with an explicit thread count, so a body may run in a block with more threads than it
// uses (the persistent batched kernel: the threads beyond NT skip the body and wait at the
// kernel's own barriers).  With NT = blockDim.x it is the same as a full block barrier.  NT must
// be a multiple of the warp size.
template <int NT>
__device__ __forceinline__ void block_sync() {
  static_assert(NT % 32 == 0, "a named barrier counts whole warps");
  asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
}

// Barrier between the stages of one transform.  A transform is owned by TT = L/PE
// consecutive threads; when TT divides 32 every transform lies inside one warp and touches
// only its own buffer, so a warp barrier (which also orders the warp's shared-memory
// accesses) replaces the block barrier.  NT: block size (the last warp may be partial).
template <int TT, int NT>
__device__ __forceinline__ void stage_sync() {
  if constexpr (TT <= 32 && 32 % TT == 0) {
    constexpr int TAIL = NT % 32;
    if constexpr (TAIL == 0) {
      __syncwarp();
    } else {
      const int wl = (int)(threadIdx.x >> 5) == NT / 32 ? TAIL : 32;
      __syncwarp(wl == 32 ? 0xffffffffu : ((1u << wl) - 1u));
    }
  } else {
    block_sync<NT>();
  }
}

// Marker: the first stage reads its inputs from the buffer (no input functor).
struct NoLoad {};

// Index of element i in the buffer one stage hands the next where a padded layout puts
// several lanes of a wavefront on one bank (see stockham_stage): every aligned group of 16
// slots rotated, by 4 ((i >> 4) mod 4) for transforms with 4 points per thread and by
// 8 ((i >> 6) mod 2) for 8 points per thread - a bijection of the unpadded indices.
template <int PE>
__device__ __forceinline__ int handoff_slot(int i) {
  if constexpr (PE == 4) return (i & ~15) | ((i + ((i >> 2) & 12)) & 15);
  else return (i & ~15) | ((i + ((i >> 3) & 8)) & 15);
}

// One Stockham stage of radix R on a length-L transform at buf (padded), current
// sub-transform length Ns.  j: this thread's index among the L/PE owners.  In the first
// stage (Ns = 1) an input functor ld(bi, m) may supply element m of transform bi instead of
// the buffer (fusing the caller's pre-pass into the stage); that stage then reads nothing
// from the buffer, so it needs no barrier between its loads and its stores.
template <typename T, int L, int PE, int R, int Ns, int DIR, int PS, int TWN, int NT, typename LD>
__device__ __forceinline__ void stockham_stage(cplx<T>* buf, int j, bool active,
                                               const TwTab<T, TWN>& tw, const cplx<T>* stab,
                                               int bi, const LD& ld) {
  constexpr int TT = L / PE;
  constexpr int NB = PE / R;
  constexpr bool FUSED = Ns == 1 && !std::is_same<LD, NoLoad>::value;
  // Padded index of i + d: when adding d cannot carry out of the low PS bits of i (d a
  // multiple of the padding interval, or every index below one interval), padi(i + d) =
  // padi(i) + d + (d >> PS), so one padded base and compile-time offsets serve all of a
  // thread's accesses in the stage.
  constexpr int SL = L / R;   // stride of a butterfly's inputs
  constexpr bool LD_OFF = SL % (1 << PS) == 0 || L <= (1 << PS);
  constexpr bool ST_OFF = Ns % (1 << PS) == 0 || Ns * R <= (1 << PS);
  // With PE = 4 or 8 points per thread the stage at Ns = PE stores (q - k) PE + k + PE r: in
  // the padded layout the lanes of a wavefront with equal k and consecutive q / PE share a
  // bank (four or two wavefronts where one would do).  Its output, read only by the stage at
  // Ns = PE^2, is stored by handoff_slot<PE> instead, under which those stores and that stage's
  // loads (consecutive indices) meet every bank once: for 8- and 16-byte elements at PE = 4,
  // for 8-byte ones at PE = 8 (16-byte ones meet no conflict there).
  constexpr bool ROTATE = PE == 4 || (PE == 8 && sizeof(T) == 4);
  constexpr bool ROT_OUT = ROTATE && Ns == PE && R == PE && Ns * R < L;
  constexpr bool ROT_IN = ROTATE && Ns == PE * PE && L > PE * PE;
  cplx<T> v[NB][R];
  if (active) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int q = j + b * TT;
      if constexpr (FUSED) {
#pragma unroll
        for (int r = 0; r < R; ++r) v[b][r] = ld(bi, q + r * SL);
      } else if constexpr (ROT_IN) {
#pragma unroll
        for (int r = 0; r < R; ++r) v[b][r] = buf[handoff_slot<PE>(q + r * SL)];
      } else if constexpr (LD_OFF) {
        const cplx<T>* p0 = buf + padi<PS>(q);
#pragma unroll
        for (int r = 0; r < R; ++r) v[b][r] = p0[r * SL + ((r * SL) >> PS)];
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) v[b][r] = buf[padi<PS>(q + r * SL)];
      }
    }
  }
  if constexpr (!FUSED) stage_sync<TT, NT>();
  if (active) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int q = j + b * TT;
      const int k = q & (Ns - 1);
      if (Ns > 1) {
        if constexpr (StageTab<T, L, PE>::USE) {
          constexpr int off = stage_offset(L, PE, Ns);
#pragma unroll
          for (int r = 1; r < R; ++r) {
            cplx<T> w = stab[off + (r - 1) * Ns + k];
            if (DIR > 0) w.y = -w.y;
            v[b][r] = cmul(v[b][r], w);
          }
        } else {
          constexpr int stride = TWN / (Ns * R);
#pragma unroll
          for (int r = 1; r < R; ++r) v[b][r] = cmul(v[b][r], twiddle<T, DIR>(tw, r * k * stride));
        }
      }
      dft_reg<T, R, DIR>(v[b]);
      const int base = (q - k) * R + k;
      if constexpr (ROT_OUT) {
#pragma unroll
        for (int r = 0; r < R; ++r) buf[handoff_slot<PE>(base + r * Ns)] = v[b][bitrev<R>(r)];
      } else if constexpr (ST_OFF) {
        cplx<T>* p0 = buf + padi<PS>(base);
#pragma unroll
        for (int r = 0; r < R; ++r) p0[r * Ns + ((r * Ns) >> PS)] = v[b][bitrev<R>(r)];
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) buf[padi<PS>(base + r * Ns)] = v[b][bitrev<R>(r)];
      }
    }
  }
  stage_sync<TT, NT>();
}

template <typename T, int L, int PE, int Ns, int DIR, int PS, int TWN, int NT, typename LD>
__device__ __forceinline__ void stockham_all(cplx<T>* buf, int j, bool active,
                                             const TwTab<T, TWN>& tw, const cplx<T>* stab,
                                             int bi, const LD& ld) {
  if constexpr (Ns < L) {
    constexpr int R = (L / Ns < PE) ? (L / Ns) : PE;
    stockham_stage<T, L, PE, R, Ns, DIR, PS, TWN, NT>(buf, j, active, tw, stab, bi, ld);
    stockham_all<T, L, PE, Ns * R, DIR, PS, TWN, NT>(buf, j, active, tw, stab, bi, NoLoad{});
  }
}

// B transforms of length L laid out at sm + b * STRIDE (padded; STRIDE = 0 means the padded
// length), all threads of the block participate (NT threads).  TWN: length of the twiddle
// table (a multiple of L); stab: this length's per-stage tables (ignored when unused);
// ld: optional input functor ld(b, m) -> element m of transform b (see stockham_stage).
// Starts with a block barrier and ends with one (the stage barriers in between are warp
// barriers when every transform lies inside one warp).
template <typename T, int L, int PE, int DIR, int NT, int TWN, int STRIDE = 0, typename LD = NoLoad>
__device__ __forceinline__ void fft_batch(cplx<T>* sm, int B, const TwTab<T, TWN>& tw, const cplx<T>* stab,
                                          const LD& ld = LD{}) {
  constexpr int PS = pad_shift<T>();
  constexpr int LP = STRIDE > 0 ? STRIDE : padded_len<L, PS>();
  constexpr int TT = L / PE;
  static_assert(NT % TT == 0, "block size must be a multiple of the threads per transform");
  constexpr int PER = NT / TT;
  const int j = threadIdx.x % TT;
  const int slot = threadIdx.x / TT;
  block_sync<NT>();
  for (int c0 = 0; c0 < B; c0 += PER) {
    const int b = c0 + slot;
    const bool active = b < B;
    stockham_all<T, L, PE, 1, DIR, PS, TWN, NT>(sm + (active ? b : 0) * LP, j, active, tw, stab, b, ld);
  }
  if constexpr (TT <= 32 && 32 % TT == 0) block_sync<NT>();
}

}  // namespace ttsh
