// ttsh_ops_impl.cuh - template launchers; included by the per-precision translation units,
// each of which defines TTSH_T (float or double), TTSH_REGISTRY (function name) and
// TTSH_SIZES (an X-macro list of the grid sizes it instantiates).
#pragma once

#include <atomic>
#include <cstring>

#include "ttsh_args.cuh"

namespace ttsh {

template <typename K>
static cudaError_t set_smem(K kernel, int bytes, std::atomic<int>& done) {
  if (done.load(std::memory_order_acquire)) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done.store(1, std::memory_order_release);
  return e;
}

// Shared memory a programmatic dependent launch of at most one block per SM reserves per
// block: more than half an SM's, so that blocks admitted early (while the previous pass
// still runs) cannot pile up two per SM and leave other SMs idle when they start.
constexpr int kSpreadSmem = 116 * 1024;

static int sm_count() {
  static std::atomic<int> sms{0};
  int v = sms.load(std::memory_order_acquire);
  if (v == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      v = 1 << 30;
    sms.store(v, std::memory_order_release);
  }
  return v;
}

// Dynamic shared memory of a step-pass launch: the pass's own, or kSpreadSmem for a
// programmatic dependent launch of at most one block per SM.
static int launch_smem(int smem, int grid, bool pdl) {
  return pdl && grid <= sm_count() && smem < kSpreadSmem ? kSpreadSmem : smem;
}

// Launch, optionally as a programmatic dependent launch (the kernel may start while the
// previous kernel in the stream is still running; it waits (griddepcontrol.wait) before it
// touches anything that kernel writes) and optionally in clusters of `cl` blocks along x.
template <typename... P, typename... V>
static cudaError_t launch_k(void (*kernel)(P...), int grid, int block, int smem, cudaStream_t s, bool pdl,
                            int cl, const V&... args) {
  if (!pdl && cl == 1) {
    kernel<<<grid, block, smem, s>>>(args...);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  int na = 0;
  if (pdl) {
    at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  if (cl > 1) {
    at[na].id = cudaLaunchAttributeClusterDimension;
    at[na].val.clusterDim.x = (unsigned)cl;
    at[na].val.clusterDim.y = 1;
    at[na].val.clusterDim.z = 1;
    ++na;
  }
  cfg.attrs = at;
  cfg.numAttrs = (unsigned)na;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <typename T, int N, int KIND, int R = default_rows<T, N>(), int PE = default_row_pe<T, N>(), int CL = 1,
          int CMP = 0>
static cudaError_t launch_row_kind(const DomainDev& d, cudaStream_t s) {
  using Geo = RowGeo<T, N, KIND, R, PE, CL, CMP>;
  static std::atomic<int> done{0};
  cudaError_t e = set_smem(row_kernel<T, N, KIND, R, PE, CL, CMP>, cmax(Geo::SMEM, kSpreadSmem), done);
  if (e != cudaSuccess) return e;
  Args<T> a = make_args<T>(d);
  CUtensorMap tm;
  memset(&tm, 0, sizeof(tm));
  constexpr int ri = R == 1 ? 0 : R == 2 ? 1 : R == 4 ? 2 : -1;
  if constexpr (Geo::TMA_OK && ri >= 0) {
    if (d.use_tma && d.tma_ok[ri] && d.err) {
      tm = d.tmapG[ri];
      a.tma = 1;
    }
  }
  const bool pdl = KIND == ROW_STEP && d.pdl;
  return launch_k(row_kernel<T, N, KIND, R, PE, CL, CMP>, N / R, Geo::NT, launch_smem(Geo::SMEM, N / R, pdl), s, pdl,
                  CL, a, tm);
}

template <typename T, int N, int MODE, int PE = default_col_pe<T, N>()>
static cudaError_t launch_col_mode(const DomainDev& d, cudaStream_t s) {
  using Geo = ColGeo<T, N, MODE, PE>;
  static std::atomic<int> done{0};
  cudaError_t e = set_smem(col_kernel<T, N, MODE, PE>, cmax(Geo::SMEM, kSpreadSmem), done);
  if (e != cudaSuccess) return e;
  // a recorded step adds one block that finishes the time-series sample
  const int extra = (MODE == COL_STEP && d.rec != nullptr) ? 1 : 0;
  const bool pdl = MODE == COL_STEP && d.pdl;
  return launch_k(col_kernel<T, N, MODE, PE>, Geo::H + extra, Geo::NT, launch_smem(Geo::SMEM, Geo::H + extra, pdl), s,
                  pdl, 1, make_args<T>(d));
}

template <typename T, int N>
static cudaError_t launch_row(int kind, const DomainDev& d, cudaStream_t s) {
  switch (kind) {
    case K_ROW_STEP: return launch_row_kind<T, N, ROW_STEP>(d, s);
    case K_ROW_FWD_VEL: return launch_row_kind<T, N, ROW_FWD_VEL>(d, s);
    case K_ROW_FWD_MASK: return launch_row_kind<T, N, ROW_FWD_MASK>(d, s);
    case K_ROW_INV_FIELDS: return launch_row_kind<T, N, ROW_INV_FIELDS>(d, s);
    case K_ROW_INV_MASK: return launch_row_kind<T, N, ROW_INV_MASK>(d, s);
    case K_ROW_INV_DIAG: return launch_row_kind<T, N, ROW_INV_DIAG>(d, s);
  }
  return cudaErrorInvalidValue;
}

template <typename T, int N>
static int row_blocks(int kind) {
  (void)kind;
  return N / default_rows<T, N>();
}

template <typename T, int N>
static cudaError_t launch_col(int mode, const DomainDev& d, cudaStream_t s) {
  switch (mode) {
    case K_COL_STEP: return launch_col_mode<T, N, COL_STEP>(d, s);
    case K_COL_PROLOGUE: return launch_col_mode<T, N, COL_PROLOGUE>(d, s);
    case K_COL_PROJECT: return launch_col_mode<T, N, COL_PROJECT>(d, s);
    case K_COL_MASK: return launch_col_mode<T, N, COL_MASK>(d, s);
    case K_COL_ADDW: return launch_col_mode<T, N, COL_ADDW>(d, s);
    case K_COL_DIV: return launch_col_mode<T, N, COL_DIV>(d, s);
  }
  return cudaErrorInvalidValue;
}

template <typename T, int N>
static cudaError_t launch_spec(const DomainDev& d, int nbins, cudaStream_t s) {
  constexpr int H = N / 4 + 1;
  spectrum_col_kernel<T, N><<<dim3((nbins + 127) / 128, H), 128, 0, s>>>(make_args<T>(d), nbins, d.colhist, d.bad);
  return cudaGetLastError();
}

template <typename T, int N, int R, int PE>
static cudaError_t launch_row_batched(const void* args, int ndom, cudaStream_t s) {
  using Geo = RowGeo<T, N, ROW_STEP, R, PE>;
  row_kernel_batched<T, N, ROW_STEP, R, PE><<<dim3(N / R, ndom), Geo::NT, Geo::SMEM, s>>>(
      static_cast<const Args<T>*>(args));
  return cudaGetLastError();
}

template <typename T, int N, int R, int PE>
static cudaError_t prepare_row_batched() {
  static std::atomic<int> done{0};
  return set_smem(row_kernel_batched<T, N, ROW_STEP, R, PE>, RowGeo<T, N, ROW_STEP, R, PE>::SMEM, done);
}

template <typename T, int N, int PE>
static cudaError_t launch_col_batched(const void* args, int ndom, cudaStream_t s) {
  using Geo = ColGeo<T, N, COL_STEP, PE>;
  col_kernel_batched<T, N, COL_STEP, PE><<<dim3(Geo::H, ndom), Geo::NT, Geo::SMEM, s>>>(
      static_cast<const Args<T>*>(args));
  return cudaGetLastError();
}

template <typename T, int N, int PE>
static cudaError_t prepare_col_batched() {
  static std::atomic<int> done{0};
  return set_smem(col_kernel_batched<T, N, COL_STEP, PE>, ColGeo<T, N, COL_STEP, PE>::SMEM, done);
}

template <typename T>
static void pack_args(const DomainDev& d, void* dst) {
  const Args<T> a = make_args<T>(d);
  memcpy(dst, &a, sizeof(a));
}

template <typename T, int N, int R, int PE, int CL = 1, int CMP = 0>
static void add_row_variant(SizeOps& o) {
  if constexpr (RowGeo<T, N, ROW_STEP, R, PE, CL, CMP>::VALID &&
                (N >= 64 || (R == default_step_rows<T, N>() && PE == default_step_row_pe<T, N>() && CL == 1 && CMP == 0))) {
    // a compact variant whose plan equals the plain one's (nothing to leave out) is the same shape
    constexpr int cmp =
        RowGeo<T, N, ROW_STEP, R, PE, CL, CMP>::SMEM != RowGeo<T, N, ROW_STEP, R, PE, CL, 0>::SMEM ? CMP : 0;
    for (int i = 0; i < o.n_row_variants; ++i)
      if (o.row_step[i].rows == R && o.row_step[i].pe == cmin(PE, N / 2) && o.row_step[i].cl == CL &&
          o.row_step[i].cmp == cmp)
        return;   // same shape
    StepVariant v{&launch_row_kind<T, N, ROW_STEP, R, PE, CL, CMP>, nullptr, nullptr, R, cmin(PE, N / 2), CL, cmp,
                  RowGeo<T, N, ROW_STEP, R, PE, CL, CMP>::TMA_OK ? 1 : 0};
    if constexpr (N <= kMaxBatchN && CL == 1 && CMP == 0) {
      v.batched = &launch_row_batched<T, N, R, PE>;
      v.prepare = &prepare_row_batched<T, N, R, PE>;
    }
    if (o.n_row_variants < kMaxVariants) o.row_step[o.n_row_variants++] = v;
  }
}

template <typename T, int N, int PE>
static void add_col_variant(SizeOps& o) {
  if constexpr (ColGeo<T, N, COL_STEP, PE>::VALID && (N >= 64 || PE == default_step_col_pe<T, N>())) {
    for (int i = 0; i < o.n_col_variants; ++i)
      if (o.col_step[i].pe == cmin(PE, N)) return;
    StepVariant v{&launch_col_mode<T, N, COL_STEP, PE>, nullptr, nullptr, 1, cmin(PE, N), 1, 0};
    if constexpr (N <= kMaxBatchN) {
      v.batched = &launch_col_batched<T, N, PE>;
      v.prepare = &prepare_col_batched<T, N, PE>;
    }
    if (o.n_col_variants < kMaxVariants) o.col_step[o.n_col_variants++] = v;
  }
}

template <typename T, int N>
static SizeOps make_ops() {
  SizeOps o;
  o.row = &launch_row<T, N>;
  o.col = &launch_col<T, N>;
  o.spec = &launch_spec<T, N>;
  o.row_blocks = &row_blocks<T, N>;
  o.n_row_variants = 0;
  o.n_col_variants = 0;
  o.args_bytes = (int)sizeof(Args<T>);
  o.pack_args = &pack_args<T>;
  add_row_variant<T, N, default_step_rows<T, N>(), default_step_row_pe<T, N>(), default_row_cluster<T, N>()>(o);
  add_col_variant<T, N, default_step_col_pe<T, N>()>(o);
  if constexpr (sizeof(T) == 4) {
    add_row_variant<T, N, 4, 16>(o);
    add_row_variant<T, N, 2, 16>(o);
    add_row_variant<T, N, 1, 16>(o);
    add_row_variant<T, N, 2, 8>(o);
    if constexpr (N >= 2048) {
      // clusters of two blocks: global segments of 2R values (large grids, where R is small)
      add_row_variant<T, N, 1, 16, 2>(o);
      add_row_variant<T, N, 2, 16, 2>(o);
    }
    if constexpr (N >= 1024 && N <= 4096) {
      // compact: in-place forward transforms, mask rows not staged: two or more blocks per SM
      add_row_variant<T, N, 2, 16, 1, 1>(o);
      add_row_variant<T, N, 1, 16, 2, 1>(o);
      add_row_variant<T, N, 1, 16, 1, 1>(o);
    }
    add_col_variant<T, N, 8>(o);
    add_col_variant<T, N, 16>(o);
    add_col_variant<T, N, 4>(o);
  } else {
    add_row_variant<T, N, 2, 8>(o);
    add_row_variant<T, N, 1, 8>(o);
    add_row_variant<T, N, 1, 4>(o);
    add_col_variant<T, N, 8>(o);
    add_col_variant<T, N, 4>(o);
  }
  return o;
}

bool TTSH_REGISTRY(int n, SizeOps* o) {
  switch (n) {
#define X(NN) \
  case NN: *o = make_ops<TTSH_T, NN>(); return true;
    TTSH_SIZES
#undef X
  }
  return false;
}

}  // namespace ttsh
