// ttsh_api.cu - host runtime behind the C ABI of include/ttsh.h.
//
// A domain owns (or borrows) one device workspace holding the spectral state, the processed
// mask, the two inter-pass buffers of the row/column step, a double staging area for host
// transfers, the diagnostics scratch and the twiddle table.  Every arithmetic step of the
// method runs in the kernels of ttsh_kernels.cuh; this file only validates arguments,
// carves the workspace, orders launches on the domain's stream and records multi-step
// loops as CUDA graphs.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <string>
#include <unordered_set>
#include <vector>

#include <nvtx3/nvToolsExt.h>   // header-only: ranges are free unless a profiler attaches

#include "ttsh.h"
#include "ttsh_kernels.cuh"
#include "ttsh_ops.h"

// Host-side NVTX range over one API call (visible to ncu --nvtx / Nsight timelines).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

namespace {

thread_local std::string g_last_error;

ttsh_status fail(ttsh_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

ttsh_status cuda_fail(cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return fail(e == cudaErrorMemoryAllocation ? TTSH_E_OOM : TTSH_E_CUDA, m);
}

#define TTSH_CUDA(call, what)                      \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

struct Layout {
  size_t what, vmean, K, G, Rr, tw, real, part, colhist, bad, out, save, rec, recctl, err, knaive, total;
};

Layout layout_for(int n, size_t elt) {
  const size_t M = n / 4, H = M + 1, NK = 2 * M + 1, NN = (size_t)n * n;
  Layout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += align_up(bytes);
    return o;
  };
  L.what = take(H * NK * 2 * elt);
  L.vmean = take(64);
  L.K = take(NN * elt);
  L.G = take(3 * H * n * 2 * elt);
  L.Rr = take(3 * H * n * 2 * elt);
  L.tw = take((size_t)n * 2 * elt);
  L.real = take(3 * NN * sizeof(double));
  // row-block diagnostic partials; also holds the 2 x 120 peak partials of ttsh_dumbbell_order
  L.part = take(std::max((size_t)n * ttsh::kDiagQ * sizeof(double), (size_t)8192));
  L.colhist = take(H * (M + 1) * sizeof(double));
  L.bad = take(64);
  L.out = take((8 + M + 1) * sizeof(double));
  L.save = take(H * NK * 2 * elt + 64);   // state copy kept by ttsh_time_kernels
  L.rec = take((size_t)n * ttsh::kDiagQ * sizeof(double));   // time-series partials (<= n row blocks)
  L.recctl = take(64);                                        // time-series write position
  L.err = take(64);                                           // device status word
  L.knaive = take(NN);                                        // binary mask as given (ttsh_init_noise)
  static_assert(sizeof(ttsh::RecCtl) <= 64, "RecCtl must fit its region");
  L.total = off;
  return L;
}

ttsh_status validate(const ttsh_params* p) {
  if (!p) return fail(TTSH_E_INVALID, "params is NULL");
  if (!is_pow2(p->n) || p->n < 16 || p->n > 8192)
    return fail(TTSH_E_INVALID, "n must be a power of two in [16, 8192]");
  if (p->precision != 32 && p->precision != 64)
    return fail(TTSH_E_INVALID, "precision must be 32 or 64");
  if (!(p->dx > 0) || !(p->dt > 0) || !std::isfinite(p->dx) || !std::isfinite(p->dt))
    return fail(TTSH_E_INVALID, "dx and dt must be positive and finite");
  const double c[5] = {p->a, p->b, p->lambda, p->gamma_v, p->gamma_w};
  for (double v : c)
    if (!std::isfinite(v)) return fail(TTSH_E_INVALID, "model coefficients must be finite");
  return TTSH_OK;
}

bool find_ops(int n, int precision, ttsh::SizeOps* o) {
  if (precision == 32) return ttsh::ops_f32_small(n, o) || ttsh::ops_f32_large(n, o);
  return ttsh::ops_f64_small(n, o) || ttsh::ops_f64_large(n, o);
}

// Twiddles W_N^m = exp(-2 pi i m / N), computed in extended precision and rounded once.
template <typename T>
std::vector<T> twiddles(int n) {
  std::vector<T> tw(2 * (size_t)n);
  const long double two_pi = 6.283185307179586476925286766559005768L;
  for (int m = 0; m < n; ++m) {
    const long double ang = two_pi * (long double)m / (long double)n;
    tw[2 * m] = (T)(double)cosl(ang);
    tw[2 * m + 1] = (T)(double)(-sinl(ang));
  }
  return tw;
}

// cuTensorMapEncodeTiled from the driver (resolved once through the runtime; no link-time
// dependency on the driver library).
typedef CUresult (*TmapEncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

TmapEncodeFn tmap_encoder() {
  static const TmapEncodeFn fn = []() -> TmapEncodeFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return reinterpret_cast<TmapEncodeFn>(p);
  }();
  return fn;
}

// Tensor maps of G ([3 (N/4+1)] rows of 2N scalars, row pitch N complex) for the row pass's
// TMA loads, one per row-block height R = 1, 2, 4 (box: 2R scalars x N/4+1 rows).  A shape
// the TMA cannot take (more than 256 rows in a box, or an R-row segment that is not a
// multiple of 16 bytes) leaves tma_ok = 0 and the row pass uses cp.async instead.
void init_tensor_maps(ttsh::DomainDev& v, int n, size_t elt) {
  const int H = n / 4 + 1;
  for (int i = 0; i < 3; ++i) {
    v.tma_ok[i] = 0;
    memset(&v.tmapG[i], 0, sizeof(v.tmapG[i]));
  }
  const TmapEncodeFn fn = tmap_encoder();
  if (!fn || H > 256) return;
  const size_t cb = 2 * elt;
  for (int i = 0; i < 3; ++i) {
    const int R = 1 << i;
    if ((R * cb) % 16 != 0 || n % R != 0) continue;
    const cuuint64_t dims[2] = {(cuuint64_t)2 * n, (cuuint64_t)3 * H};
    const cuuint64_t strides[1] = {(cuuint64_t)n * cb};
    const cuuint32_t box[2] = {(cuuint32_t)(2 * R), (cuuint32_t)H};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r = fn(&v.tmapG[i], elt == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2,
                          v.G, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    v.tma_ok[i] = r == CUDA_SUCCESS ? 1 : 0;
  }
}

}  // namespace

struct ttsh_domain {
  ttsh_params p;
  int n, M, H, NK;
  size_t elt;
  cudaStream_t stream;
  cudaStream_t capture;     // private stream used only to record graphs
  void* ws;
  bool owns_ws;
  Layout lay;
  ttsh::DomainDev dev;
  ttsh::SizeOps ops;
  int64_t steps;
  cudaGraphExec_t graph;
  int graph_len;
  int rv, cv;   // selected tile shapes of the row and column step kernels
  // temporal power spectral density accumulators (ttsh_psd_*)
  int psd_nfreq = 0;
  double* psd_omega = nullptr;   // nfreq angular frequencies
  double2* psd_acc = nullptr;    // [2][nfreq][H*NK]: sums with exp(-i W t) and exp(+i W t)
  double* psd_S = nullptr;       // nfreq results
  // time-series recording (ttsh_step_record): cached graph of `rec_len` steps with a sample
  // every `rec_every` steps, valid for the centre and plan below (the destination is read
  // from device memory set at each call)
  cudaGraphExec_t rec_graph = nullptr;
  int rec_len = 0, rec_every = 0, rec_rv = -1, rec_cv = -1;
  double rec_cx = 0.0, rec_cy = 0.0;
};

namespace ttsh {
// Test hook of the failure path: one block waits on an mbarrier phase that nothing completes
// (no arrival is ever made), bounded by limit_ns; the wait runs out and sets the status word.
__global__ void expire_wait_kernel(int* err, unsigned long long limit_ns) {
  __shared__ __align__(8) unsigned long long bar;
  const unsigned a = (unsigned)__cvta_generic_to_shared(&bar);
  if (threadIdx.x == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait_bounded(a, 0, limit_ns)) atomicExch(err, 1);
}
}  // namespace ttsh

namespace {

constexpr int kGraphLen = 64;   // steps recorded per graph replay

ttsh_status run_row(ttsh_domain* d, int kind, cudaStream_t s) {
  cudaError_t e = d->ops.row(kind, d->dev, s);
  if (e != cudaSuccess) return cuda_fail(e, "row kernel launch");
  return TTSH_OK;
}

ttsh_status run_col(ttsh_domain* d, int mode, cudaStream_t s) {
  cudaError_t e = d->ops.col(mode, d->dev, s);
  if (e != cudaSuccess) return cuda_fail(e, "column kernel launch");
  return TTSH_OK;
}

ttsh_status one_step(ttsh_domain* d, cudaStream_t s) {
  cudaError_t e = d->ops.row_step[d->rv].fn(d->dev, s);
  if (e != cudaSuccess) return cuda_fail(e, "row pass launch");
  e = d->ops.col_step[d->cv].fn(d->dev, s);
  if (e != cudaSuccess) return cuda_fail(e, "column pass launch");
  return TTSH_OK;
}

// Mean duration of one launch of fn, from CUDA events around graph replays (the launches are
// recorded in graphs of up to 128 so that host launch overhead is not timed).
ttsh_status time_launches(ttsh_domain* d, ttsh::StepFn fn, int iters, double* ms) {
  cudaError_t e = fn(d->dev, d->stream);   // sets kernel attributes outside capture
  if (e != cudaSuccess) return cuda_fail(e, "timing warm-up");
  const int per = iters < 128 ? iters : 128;
  const int reps = (iters + per - 1) / per;
  TTSH_CUDA(cudaStreamSynchronize(d->stream), "timing warm-up");
  TTSH_CUDA(cudaStreamBeginCapture(d->capture, cudaStreamCaptureModeThreadLocal), "begin capture");
  for (int i = 0; i < per && e == cudaSuccess; ++i) e = fn(d->dev, d->capture);
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(d->capture, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(e != cudaSuccess ? e : e2, "timing capture");
  }
  cudaGraphExec_t ge = nullptr;
  e = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "timing graph instantiate");
  cudaEvent_t ev[2];
  cudaEventCreate(&ev[0]);
  cudaEventCreate(&ev[1]);
  e = cudaGraphLaunch(ge, d->stream);   // warm
  if (e == cudaSuccess) e = cudaEventRecord(ev[0], d->stream);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) e = cudaGraphLaunch(ge, d->stream);
  if (e == cudaSuccess) e = cudaEventRecord(ev[1], d->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ev[0], ev[1]);
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  cudaGraphExecDestroy(ge);
  if (e != cudaSuccess) return cuda_fail(e, "kernel timing");
  *ms = (double)t / ((double)reps * per);
  return TTSH_OK;
}

// Mean duration of one whole step (row pass then column pass of the current plan and launch
// mode), from CUDA events around replays of a graph of up to 64 steps.  Advances the state:
// callers save and restore it.
ttsh_status time_steps(ttsh_domain* d, int iters, double* ms) {
  ttsh_status st = one_step(d, d->stream);   // sets kernel attributes outside capture
  if (st != TTSH_OK) return st;
  const int per = iters < 64 ? iters : 64;
  const int reps = (iters + per - 1) / per;
  TTSH_CUDA(cudaStreamSynchronize(d->stream), "timing warm-up");
  TTSH_CUDA(cudaStreamBeginCapture(d->capture, cudaStreamCaptureModeThreadLocal), "begin capture");
  for (int i = 0; i < per && st == TTSH_OK; ++i) st = one_step(d, d->capture);
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(d->capture, &g);
  if (st != TTSH_OK || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return st != TTSH_OK ? st : cuda_fail(e2, "timing capture");
  }
  cudaGraphExec_t ge = nullptr;
  cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "timing graph instantiate");
  cudaEvent_t ev[2];
  cudaEventCreate(&ev[0]);
  cudaEventCreate(&ev[1]);
  e = cudaGraphLaunch(ge, d->stream);   // warm
  if (e == cudaSuccess) e = cudaEventRecord(ev[0], d->stream);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) e = cudaGraphLaunch(ge, d->stream);
  if (e == cudaSuccess) e = cudaEventRecord(ev[1], d->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ev[0], ev[1]);
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  cudaGraphExecDestroy(ge);
  if (e != cudaSuccess) return cuda_fail(e, "step timing");
  *ms = (double)t / ((double)reps * per);
  return TTSH_OK;
}

// Save / restore the spectral state around timing runs of the column pass.
ttsh_status save_state(ttsh_domain* d) {
  const size_t wbytes = (size_t)d->H * d->NK * 2 * d->elt;
  char* save = static_cast<char*>(d->ws) + d->lay.save;
  TTSH_CUDA(cudaMemcpyAsync(save, d->dev.what, wbytes, cudaMemcpyDeviceToDevice, d->stream), "save state");
  TTSH_CUDA(cudaMemcpyAsync(save + wbytes, d->dev.vmean, 64, cudaMemcpyDeviceToDevice, d->stream), "save mean");
  return TTSH_OK;
}

ttsh_status restore_state(ttsh_domain* d) {
  const size_t wbytes = (size_t)d->H * d->NK * 2 * d->elt;
  char* save = static_cast<char*>(d->ws) + d->lay.save;
  TTSH_CUDA(cudaMemcpyAsync(d->dev.what, save, wbytes, cudaMemcpyDeviceToDevice, d->stream), "restore state");
  TTSH_CUDA(cudaMemcpyAsync(d->dev.vmean, save + wbytes, 64, cudaMemcpyDeviceToDevice, d->stream), "restore mean");
  ttsh_status st = run_col(d, ttsh::K_COL_PROLOGUE, d->stream);
  if (st != TTSH_OK) return st;
  TTSH_CUDA(cudaStreamSynchronize(d->stream), "restore state");
  return TTSH_OK;
}

ttsh_status sync(ttsh_domain* d, const char* what) {
  TTSH_CUDA(cudaStreamSynchronize(d->stream), what);
  return TTSH_OK;
}

ttsh_status build_graph(ttsh_domain* d) {
  // The capture runs on a private stream; replays are launched on the domain's stream.
  TTSH_CUDA(cudaStreamBeginCapture(d->capture, cudaStreamCaptureModeThreadLocal), "begin capture");
  ttsh_status st = TTSH_OK;
  for (int i = 0; i < kGraphLen && st == TTSH_OK; ++i) st = one_step(d, d->capture);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(d->capture, &g);
  if (st != TTSH_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(e, "end capture");
  e = cudaGraphInstantiate(&d->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    d->graph = nullptr;
    return cuda_fail(e, "graph instantiate");
  }
  d->graph_len = kGraphLen;
  return TTSH_OK;
}

// Device status word: a kernel whose bounded wait ran out set it; report it once.
ttsh_status check_status(ttsh_domain* d) {
  // on the domain's stream: kernels there may run on a non-blocking stream, which the legacy
  // default stream does not order against
  int h = 0;
  TTSH_CUDA(cudaMemcpyAsync(&h, d->dev.err, sizeof(int), cudaMemcpyDeviceToHost, d->stream), "read status word");
  TTSH_CUDA(cudaStreamSynchronize(d->stream), "read status word");
  if (h) {
    TTSH_CUDA(cudaMemsetAsync(d->dev.err, 0, sizeof(int), d->stream), "clear status word");
    return fail(TTSH_E_TIMEOUT, "a bounded wait in a kernel ran out (results of the affected steps are not valid)");
  }
  return TTSH_OK;
}

ttsh_status project_staged(ttsh_domain* d) {
  ttsh_status st = run_row(d, ttsh::K_ROW_FWD_VEL, d->stream);
  if (st != TTSH_OK) return st;
  st = run_col(d, ttsh::K_COL_PROJECT, d->stream);
  if (st != TTSH_OK) return st;
  d->steps = 0;
  return sync(d, "set_velocity");
}

template <typename T>
void to_host_double(const std::vector<T>& src, double* dst) {
  for (size_t i = 0; i < src.size(); ++i) dst[i] = (double)src[i];
}

}  // namespace

namespace ttsh {

__global__ void diag_reduce_kernel(const double* __restrict__ part, int nblocks, double* out) {
  __shared__ double red[kDiagQ][256];
  const int t = threadIdx.x;
  double acc[kDiagQ] = {0, 0, 0, 0, 0};
  for (int i = t; i < nblocks; i += 256)
    for (int q = 0; q < kDiagQ; ++q) acc[q] += part[(size_t)i * kDiagQ + q];
  for (int q = 0; q < kDiagQ; ++q) red[q][t] = acc[q];
  __syncthreads();
  for (int s = 128; s >= 1; s >>= 1) {
    if (t < s)
      for (int q = 0; q < kDiagQ; ++q) red[q][t] += red[q][t + s];
    __syncthreads();
  }
  if (t < kDiagQ) out[t] = red[t][0];
}

__global__ void spectrum_reduce_kernel(const double* __restrict__ colhist, int ncols, int nbins,
                                       double scale, double* __restrict__ out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nbins) return;
  double acc = 0.0;
  for (int c = 0; c < ncols; ++c) acc += colhist[(size_t)c * nbins + s];
  out[s] = acc * scale;
}

void set_last_error(const char* msg) { g_last_error = msg; }

void set_last_error(const char* what, cudaError_t e) { cuda_fail(e, what); }

cudaError_t launch_diag_reduce(const double* part, int nblocks, double* out, cudaStream_t s) {
  diag_reduce_kernel<<<1, 256, 0, s>>>(part, nblocks, out);
  return cudaGetLastError();
}

cudaError_t launch_spectrum_reduce(const double* colhist, int ncols, int nbins, double scale,
                                   double* out, cudaStream_t s) {
  spectrum_reduce_kernel<<<(nbins + 127) / 128, 128, 0, s>>>(colhist, ncols, nbins, scale, out);
  return cudaGetLastError();
}

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) in counter form: output i of the stream
// started at `seed` is the 64-bit finaliser applied to seed + (i + 1) * 0x9E3779B97F4A7C15.
__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed, unsigned long long i) {
  unsigned long long z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// The initial velocity of the paper's runs, a "random initial state" (Sec. III.A): at every
// point inside the domain (K_naive = 0) v_x and v_y are i.i.d. uniform on [-A, A), v_x from
// draw 2p and v_y from draw 2p + 1 of point p = y N + x; a draw z gives u = (z >> 11) 2^-53
// in [0, 1) and A (2u - 1).  Masked points get 0.  Written to the double staging planes 0
// and 1, which the projection of the initial state reads; explicit roundings, so the values
// are the same bits as any other implementation of this definition in double precision.
__global__ void noise_kernel(double* __restrict__ real, const unsigned char* __restrict__ knaive, long long nn,
                             unsigned long long seed, double amp) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < nn; p += stride) {
    double vx = 0.0, vy = 0.0;
    if (knaive[p] == 0) {
      const unsigned long long i = 2ull * (unsigned long long)p;
      const double ux = (double)(splitmix64_at(seed, i) >> 11) * 0x1.0p-53;
      const double uy = (double)(splitmix64_at(seed, i + 1) >> 11) * 0x1.0p-53;
      vx = __dmul_rn(amp, __dsub_rn(__dmul_rn(2.0, ux), 1.0));
      vy = __dmul_rn(amp, __dsub_rn(__dmul_rn(2.0, uy), 1.0));
    }
    real[p] = vx;
    real[nn + p] = vy;
  }
}

__global__ void record_begin_kernel(RecCtl* c, long long base, double* series, long long capacity,
                                    int every, int nblocks, double inv2n2) {
  c->count = 0;
  c->base = base;
  c->series = series;
  c->capacity = capacity;
  c->every = every;
  c->nblocks = nblocks;
  c->inv2n2 = inv2n2;
  c->overflow = 0;
}

}  // namespace ttsh


namespace ttsh {
const DomainDev* domain_dev(const ttsh_domain* d) { return &d->dev; }
cudaStream_t domain_stream(const ttsh_domain* d) { return d->stream; }
int domain_precision(const ttsh_domain* d) { return d->p.precision; }
int domain_n(const ttsh_domain* d) { return d->n; }
double domain_dx(const ttsh_domain* d) { return d->p.dx; }
int domain_fields_to_staging(ttsh_domain* d) { return run_row(d, K_ROW_INV_FIELDS, d->stream); }
void domain_add_steps(ttsh_domain* d, int64_t n) { d->steps += n; }
int domain_add_vorticity_from_staging(ttsh_domain* d) {
  ttsh_status st = run_row(d, K_ROW_FWD_MASK, d->stream);   // one real field forward
  if (st != TTSH_OK) return st;
  return run_col(d, K_COL_ADDW, d->stream);
}
double domain_dt(const ttsh_domain* d) { return d->p.dt; }
int domain_refresh(ttsh_domain* d) { return run_col(d, K_COL_PROLOGUE, d->stream); }
int domain_refresh_on(ttsh_domain* d, cudaStream_t s) { return run_col(d, K_COL_PROLOGUE, s); }

// A second domain with the same parameters, processed mask, twiddles, plan, launch mode,
// stream and state as src (device-to-device copies; the library allocates its workspace).
int domain_clone(const ttsh_domain* src, ttsh_domain** out) {
  *out = nullptr;
  ttsh_domain* d = new ttsh_domain();
  d->p = src->p;
  d->n = src->n;
  d->M = src->M;
  d->H = src->H;
  d->NK = src->NK;
  d->elt = src->elt;
  d->stream = src->stream;
  d->capture = nullptr;
  d->ops = src->ops;
  d->steps = src->steps;
  d->graph = nullptr;
  d->graph_len = 0;
  d->rv = src->rv;
  d->cv = src->cv;
  d->lay = src->lay;
  d->owns_ws = true;
  d->ws = nullptr;
  auto cleanup = [&](ttsh_status s) {
    ttsh_destroy_domain(d);
    return (int)s;
  };
  cudaError_t e = cudaMalloc(&d->ws, d->lay.total);
  if (e != cudaSuccess) {
    d->ws = nullptr;
    return cleanup(cuda_fail(e, "workspace allocation"));
  }
  e = cudaStreamCreateWithFlags(&d->capture, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "capture stream"));
  d->dev = src->dev;   // constants, centre, launch mode; pointers rebased below
  char* base = static_cast<char*>(d->ws);
  DomainDev& v = d->dev;
  v.what = base + d->lay.what;
  v.vmean = base + d->lay.vmean;
  v.K = base + d->lay.K;
  v.G = base + d->lay.G;
  v.Rr = base + d->lay.Rr;
  v.tw = base + d->lay.tw;
  v.real = reinterpret_cast<double*>(base + d->lay.real);
  v.part = reinterpret_cast<double*>(base + d->lay.part);
  v.colhist = reinterpret_cast<double*>(base + d->lay.colhist);
  v.bad = reinterpret_cast<int*>(base + d->lay.bad);
  v.out = reinterpret_cast<double*>(base + d->lay.out);
  v.rec = nullptr;
  v.recctl = nullptr;
  v.err = reinterpret_cast<int*>(base + d->lay.err);
  v.knaive = reinterpret_cast<unsigned char*>(base + d->lay.knaive);
  init_tensor_maps(v, d->n, d->elt);
  const size_t NN = (size_t)d->n * d->n;
  const size_t wbytes = (size_t)d->H * d->NK * 2 * d->elt;
  e = cudaMemsetAsync(v.err, 0, 64, d->stream);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "status word"));
  e = cudaMemcpyAsync(v.K, src->dev.K, NN * d->elt, cudaMemcpyDeviceToDevice, d->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(v.tw, src->dev.tw, (size_t)d->n * 2 * d->elt, cudaMemcpyDeviceToDevice, d->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(v.what, src->dev.what, wbytes, cudaMemcpyDeviceToDevice, d->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(v.vmean, src->dev.vmean, 64, cudaMemcpyDeviceToDevice, d->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(v.knaive, src->dev.knaive, NN, cudaMemcpyDeviceToDevice, d->stream);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "clone copies"));
  ttsh_status st = run_col(d, K_COL_PROLOGUE, d->stream);
  if (st != TTSH_OK) return cleanup(st);
  *out = d;
  return TTSH_OK;
}

// Spectral restriction of a fine state onto a coarse grid of the same box: the coarse
// unitary coefficients are the fine ones times Nc/Nf on the coarse 1/2-rule disc.
template <typename T>
__global__ void restrict_kernel(const cplx<T>* __restrict__ wf, const T* __restrict__ vf, int nf,
                                cplx<T>* __restrict__ wc, T* __restrict__ vc, int nc) {
  const int Mf = nf / 4, NKf = 2 * Mf + 1, Mc = nc / 4, NKc = 2 * Mc + 1, Hc = Mc + 1;
  const T s = (T)nc / (T)nf;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Hc * NKc) return;
  const int kx = i / NKc, j = i % NKc;
  const int ky = j <= Mc ? j : j - NKc;
  const int jf = ky >= 0 ? ky : ky + NKf;
  cplx<T> w = wf[(size_t)kx * NKf + jf];
  if (kx * kx + ky * ky > Mc * Mc) w = mk<T>(0, 0);
  wc[i] = w * s;
  if (i == 0) {
    vc[0] = vf[0] * s;
    vc[1] = vf[1] * s;
  }
}

// ---- dynamics diagnostics: temporal PSD (Eq. PSD) and the dumbbell order parameter ----
// PSD: S(W) = N^-2 sum_x |sum_t omega(x,t) e^{-iWt}|^2 = N^-2 sum_k |sum_t omega^(k,t) e^{-iWt}|^2
// (Parseval, unitary DFT).  Only mx >= 0 is stored; the mode -k of the accumulated sum is
// conj(sum_t omega^(k,t) e^{+iWt}), so for mx > 0 both sums are kept.
template <typename T>
__global__ void psd_accumulate_kernel(const cplx<T>* __restrict__ what, int nmodes, const double* __restrict__ om,
                                      double t, double2* __restrict__ acc, int nfreq) {
  __shared__ double cs[2];
  const int j = blockIdx.y;
  if (threadIdx.x == 0) sincos(om[j] * t, &cs[1], &cs[0]);
  __syncthreads();
  const double c = cs[0], sn = cs[1];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nmodes; i += gridDim.x * blockDim.x) {
    const double wr = (double)what[i].x, wi = (double)what[i].y;
    double2& a = acc[(size_t)j * nmodes + i];
    double2& b = acc[((size_t)nfreq + j) * nmodes + i];
    a.x += wr * c + wi * sn;   // (wr + i wi)(c - i s)
    a.y += wi * c - wr * sn;
    b.x += wr * c - wi * sn;   // (wr + i wi)(c + i s)
    b.y += wi * c + wr * sn;
  }
}

__global__ void psd_result_kernel(const double2* __restrict__ acc, int NK, int nmodes, int nfreq, double scale,
                                  double* __restrict__ S) {
  __shared__ double red[256];
  const int j = blockIdx.x, t = threadIdx.x;
  double sum = 0.0;
  for (int i = t; i < nmodes; i += 256) {
    const double2 a = acc[(size_t)j * nmodes + i];
    sum += a.x * a.x + a.y * a.y;
    if (i >= NK) {   // mx > 0: the mirrored mode
      const double2 b = acc[((size_t)nfreq + j) * nmodes + i];
      sum += b.x * b.x + b.y * b.y;
    }
  }
  red[t] = sum;
  __syncthreads();
  for (int s2 = 128; s2 >= 1; s2 >>= 1) {
    if (t < s2) red[t] += red[t + s2];
    __syncthreads();
  }
  if (t == 0) S[j] = red[0] * scale;
}

// Psi_2: per-block argmax of |omega| inside the closed discs around the two cavity centres
// (ties to the smaller row-major index), then a single-block final reduction.
struct Peak {
  double absval, val;
  long long idx;
};
__device__ __forceinline__ bool better(const Peak& a, const Peak& b) {
  return a.absval > b.absval || (a.absval == b.absval && a.idx < b.idx);
}

__global__ void dumbbell_partial_kernel(const double* __restrict__ w, int n, double dx, double c0x, double c0y,
                                        double c1x, double c1y, double r2, Peak* __restrict__ part) {
  __shared__ Peak red[2][256];
  Peak best[2] = {{-1.0, 0.0, -1}, {-1.0, 0.0, -1}};
  const long long total = (long long)n * n;
  for (long long p = blockIdx.x * 256LL + threadIdx.x; p < total; p += 256LL * gridDim.x) {
    const int ix = (int)(p % n), iy = (int)(p / n);
    const double x = (double)(ix - n / 2) * dx, y = (double)(iy - n / 2) * dx;
    const double v = w[p];
    const double cx[2] = {c0x, c1x}, cy[2] = {c0y, c1y};
    for (int c = 0; c < 2; ++c) {
      const double ddx = __dsub_rn(x, cx[c]), ddy = __dsub_rn(y, cy[c]);
      const double d2 = __dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy));
      if (d2 <= r2) {
        const Peak cand{fabs(v), v, p};
        if (better(cand, best[c])) best[c] = cand;
      }
    }
  }
  red[0][threadIdx.x] = best[0];
  red[1][threadIdx.x] = best[1];
  __syncthreads();
  for (int s2 = 128; s2 >= 1; s2 >>= 1) {
    if (threadIdx.x < s2)
      for (int c = 0; c < 2; ++c)
        if (better(red[c][threadIdx.x + s2], red[c][threadIdx.x])) red[c][threadIdx.x] = red[c][threadIdx.x + s2];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = red[0][0];
    part[2 * blockIdx.x + 1] = red[1][0];
  }
}

__global__ void dumbbell_final_kernel(const Peak* __restrict__ part, int nblocks, double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  Peak b[2] = {{-1.0, 0.0, -1}, {-1.0, 0.0, -1}};
  for (int i = 0; i < nblocks; ++i)
    for (int c = 0; c < 2; ++c)
      if (better(part[2 * i + c], b[c])) b[c] = part[2 * i + c];
  const double a = b[0].val, bb = b[1].val;
  const double den = fabs(a) + fabs(bb);
  out[0] = den > 0 ? fabs(a + bb) / den : 0.0;
  out[1] = a;
  out[2] = bb;
  out[3] = (b[0].idx < 0 || b[1].idx < 0) ? 1.0 : 0.0;   // an empty region
}
}  // namespace ttsh

// ---------------------------------------------------------------------------------------
// Batched stepping: domains grouped by (precision, n, plan); one launch per pass per group
// advances every domain of the group (blockIdx.y = domain).  Groups are independent, so each
// runs its own launch chain in a parallel branch of one CUDA graph.
// ---------------------------------------------------------------------------------------
struct BatchGroup {
  int precision = 0, n = 0, rv = 0, cv = 0;
  std::vector<ttsh_domain*> doms;
  void* args_dev = nullptr;
  const ttsh::StepVariant* row = nullptr;
  const ttsh::StepVariant* col = nullptr;
  cudaStream_t branch = nullptr;
  cudaEvent_t join = nullptr;
};

struct ttsh_batch {
  std::vector<BatchGroup> groups;
  std::vector<ttsh_domain*> all;
  cudaStream_t stream = nullptr;
  cudaStream_t capture = nullptr;
  cudaEvent_t fork = nullptr;
  cudaEvent_t order = nullptr;       // orders each domain's own stream before the batch's work
  cudaGraphExec_t graph = nullptr;   // kBatchGraphLen steps
  int graph_len = 0;
  cudaGraphExec_t tail = nullptr;    // the last call's remainder (tail_len < kBatchGraphLen steps)
  int tail_len = 0;
  // persistent mode: one launch per ttsh_batch_step call for every domain (one precision,
  // n <= max_n, default tile shapes); see ttsh_persist.cuh
  bool can_persist = false;
  bool persistent = false;
  ttsh::PersistOps pops{};
  void* pdoms = nullptr;               // device domain table
  void* pitems = nullptr;              // device work-item list of one step
  void* ptest = nullptr;               // one-item list of ttsh_batch_test_stalled_wait
  unsigned long long* pctl = nullptr;  // device control block: 2 + 2 ndom counters
  int pips = 0, pgrid = 0;
};

namespace {

constexpr int kBatchGraphLen = 32;

ttsh_status batch_group_steps(BatchGroup& g, int nsteps, cudaStream_t s) {
  const int nd = (int)g.doms.size();
  for (int i = 0; i < nsteps; ++i) {
    cudaError_t e = g.row->batched(g.args_dev, nd, s);
    if (e == cudaSuccess) e = g.col->batched(g.args_dev, nd, s);
    if (e != cudaSuccess) return cuda_fail(e, "batched launch");
  }
  return TTSH_OK;
}

// Graph of `len` steps of every group, the groups as parallel branches.
ttsh_status batch_build_graph(ttsh_batch* b, int len, cudaGraphExec_t* out) {
  TTSH_CUDA(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal), "begin capture");
  ttsh_status st = TTSH_OK;
  cudaError_t e = cudaEventRecord(b->fork, b->capture);
  for (size_t i = 0; i < b->groups.size() && e == cudaSuccess && st == TTSH_OK; ++i) {
    BatchGroup& g = b->groups[i];
    e = cudaStreamWaitEvent(g.branch, b->fork, 0);
    if (e == cudaSuccess) st = batch_group_steps(g, len, g.branch);
    if (e == cudaSuccess && st == TTSH_OK) e = cudaEventRecord(g.join, g.branch);
    if (e == cudaSuccess && st == TTSH_OK) e = cudaStreamWaitEvent(b->capture, g.join, 0);
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(b->capture, &graph);
  if (st != TTSH_OK || e != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    if (st != TTSH_OK) return st;
    return cuda_fail(e != cudaSuccess ? e : e2, "batch capture");
  }
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    *out = nullptr;
    return cuda_fail(e, "batch graph instantiate");
  }
  return TTSH_OK;
}

}  // namespace

namespace {

// One step whose row pass also writes the time-series partials; an extra block of its column
// pass appends the sample.
ttsh_status record_step(ttsh_domain* d, cudaStream_t s) {
  char* base = static_cast<char*>(d->ws);
  ttsh::DomainDev dv = d->dev;
  dv.rec = reinterpret_cast<double*>(base + d->lay.rec);
  dv.recctl = base + d->lay.recctl;
  dv.cx = d->rec_cx;
  dv.cy = d->rec_cy;
  cudaError_t e = d->ops.row_step[d->rv].fn(dv, s);
  if (e != cudaSuccess) return cuda_fail(e, "recorded row pass launch");
  e = d->ops.col_step[d->cv].fn(dv, s);
  if (e != cudaSuccess) return cuda_fail(e, "recorded column pass launch");
  return TTSH_OK;
}

void drop_record_graph(ttsh_domain* d) {
  if (d->rec_graph) cudaGraphExecDestroy(d->rec_graph);
  d->rec_graph = nullptr;
  d->rec_len = 0;
}

// Graph of rec_len = every * floor(kGraphLen / every) steps with a sample at every
// `every`-th step, starting with one.
ttsh_status build_record_graph(ttsh_domain* d) {
  const int len = d->rec_every * (kGraphLen / d->rec_every);
  TTSH_CUDA(cudaStreamBeginCapture(d->capture, cudaStreamCaptureModeThreadLocal), "begin capture");
  ttsh_status st = TTSH_OK;
  for (int i = 0; i < len && st == TTSH_OK; ++i)
    st = (i % d->rec_every == 0) ? record_step(d, d->capture) : one_step(d, d->capture);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(d->capture, &g);
  if (st != TTSH_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(e, "end capture");
  e = cudaGraphInstantiate(&d->rec_graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    d->rec_graph = nullptr;
    return cuda_fail(e, "graph instantiate");
  }
  d->rec_len = len;
  return TTSH_OK;
}

}  // namespace

extern "C" {

void ttsh_default_params(ttsh_params* p) {
  if (!p) return;
  p->a = 0.5;
  p->b = 1.6;
  p->lambda = 9.0;
  p->gamma_v = 40.0;
  p->gamma_w = 4.0;
  p->dx = 0.005;
  p->dt = 0.01;
  p->n = 8192;
  p->precision = 32;
}

size_t ttsh_workspace_bytes(const ttsh_params* p) {
  if (validate(p) != TTSH_OK) return 0;
  return layout_for(p->n, p->precision == 32 ? sizeof(float) : sizeof(double)).total;
}

ttsh_status ttsh_create_domain(const uint8_t* mask, const ttsh_params* p, void* workspace,
                               void* stream, ttsh_domain** out) {
  g_last_error.clear();
  if (!out) return fail(TTSH_E_INVALID, "out is NULL");
  *out = nullptr;
  if (!mask) return fail(TTSH_E_INVALID, "mask is NULL");
  ttsh_status st = validate(p);
  if (st != TTSH_OK) return st;
  if (workspace && (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0)
    return fail(TTSH_E_INVALID, "workspace must be 256-byte aligned");
  ttsh::SizeOps ops;
  if (!find_ops(p->n, p->precision, &ops))
    return fail(TTSH_E_UNSUPPORTED, "no kernels for this (n, precision): double precision supports n <= 4096");

  ttsh_domain* d = new ttsh_domain();
  d->p = *p;
  d->n = p->n;
  d->M = p->n / 4;
  d->H = d->M + 1;
  d->NK = 2 * d->M + 1;
  d->elt = p->precision == 32 ? sizeof(float) : sizeof(double);
  d->stream = static_cast<cudaStream_t>(stream);
  d->capture = nullptr;
  d->ops = ops;
  d->steps = 0;
  d->graph = nullptr;
  d->graph_len = 0;
  d->rv = 0;
  d->cv = 0;
  d->lay = layout_for(d->n, d->elt);
  d->owns_ws = workspace == nullptr;
  d->ws = workspace;
  auto cleanup = [&](ttsh_status s) {
    ttsh_destroy_domain(d);
    return s;
  };
  if (d->owns_ws) {
    cudaError_t e = cudaMalloc(&d->ws, d->lay.total);
    if (e != cudaSuccess) {
      d->ws = nullptr;
      return cleanup(cuda_fail(e, "workspace allocation"));
    }
  }
  {
    cudaError_t e = cudaStreamCreateWithFlags(&d->capture, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "capture stream"));
  }
  char* base = static_cast<char*>(d->ws);
  ttsh::DomainDev& v = d->dev;
  v.what = base + d->lay.what;
  v.vmean = base + d->lay.vmean;
  v.K = base + d->lay.K;
  v.G = base + d->lay.G;
  v.Rr = base + d->lay.Rr;
  v.tw = base + d->lay.tw;
  v.real = reinterpret_cast<double*>(base + d->lay.real);
  v.part = reinterpret_cast<double*>(base + d->lay.part);
  v.colhist = reinterpret_cast<double*>(base + d->lay.colhist);
  v.bad = reinterpret_cast<int*>(base + d->lay.bad);
  v.out = reinterpret_cast<double*>(base + d->lay.out);
  v.a = p->a;
  v.b = p->b;
  v.lam = p->lambda;
  v.gv = p->gamma_v;
  v.gw = p->gamma_w;
  v.dx = p->dx;
  v.dt = p->dt;
  v.cx = 0.0;
  v.cy = 0.0;
  v.n = p->n;
  v.rec = nullptr;
  v.recctl = nullptr;
  v.pdl = 0;
  v.use_tma = 0;
  v.err = reinterpret_cast<int*>(base + d->lay.err);
  v.knaive = reinterpret_cast<unsigned char*>(base + d->lay.knaive);
  init_tensor_maps(v, d->n, d->elt);
  {
    cudaError_t e = cudaMemsetAsync(v.err, 0, 64, d->stream);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "status word"));
  }

  const size_t NN = (size_t)d->n * d->n;
  cudaStream_t s = d->stream;
  // twiddle table
  if (d->elt == sizeof(float)) {
    std::vector<float> tw = twiddles<float>(d->n);
    cudaError_t e = cudaMemcpyAsync(v.tw, tw.data(), tw.size() * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "twiddle upload"));
  } else {
    std::vector<double> tw = twiddles<double>(d->n);
    cudaError_t e = cudaMemcpyAsync(v.tw, tw.data(), tw.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "twiddle upload"));
  }
  // Algorithm 2 on the device: K_naive (0/1) -> DFT -> |m|^2 <= (N/8)^2 -> iDFT -> square.
  {
    std::vector<double> kn(NN);
    std::vector<unsigned char> kb(NN);
    for (size_t i = 0; i < NN; ++i) {
      kn[i] = mask[i] ? 1.0 : 0.0;
      kb[i] = mask[i] ? 1 : 0;
    }
    cudaError_t e = cudaMemcpyAsync(v.real, kn.data(), NN * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(v.knaive, kb.data(), NN, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "mask upload"));
  }
  if ((st = run_row(d, ttsh::K_ROW_FWD_MASK, s)) != TTSH_OK) return cleanup(st);
  if ((st = run_col(d, ttsh::K_COL_MASK, s)) != TTSH_OK) return cleanup(st);
  if ((st = run_row(d, ttsh::K_ROW_INV_MASK, s)) != TTSH_OK) return cleanup(st);
  // zero state, consistent inter-pass buffers
  {
    cudaError_t e = cudaMemsetAsync(v.what, 0, (size_t)d->H * d->NK * 2 * d->elt, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(v.vmean, 0, 64, s);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "state init"));
  }
  if ((st = run_col(d, ttsh::K_COL_PROLOGUE, s)) != TTSH_OK) return cleanup(st);
  if ((st = sync(d, "create_domain")) != TTSH_OK) return cleanup(st);
  *out = d;
  return TTSH_OK;
}

void ttsh_destroy_domain(ttsh_domain* d) {
  if (!d) return;
  if (d->psd_omega) cudaFree(d->psd_omega);
  if (d->psd_acc) cudaFree(d->psd_acc);
  if (d->psd_S) cudaFree(d->psd_S);
  if (d->graph) cudaGraphExecDestroy(d->graph);
  if (d->rec_graph) cudaGraphExecDestroy(d->rec_graph);
  if (d->capture) cudaStreamDestroy(d->capture);
  if (d->owns_ws && d->ws) cudaFree(d->ws);
  delete d;
}

ttsh_status ttsh_set_stream(ttsh_domain* d, void* stream) {
  if (!d) return fail(TTSH_E_INVALID, "domain is NULL");
  cudaStream_t ns = static_cast<cudaStream_t>(stream);
  if (ns != d->stream) {
    // work already queued on the old stream comes first (device-side wait)
    cudaEvent_t ev = nullptr;
    TTSH_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "stream switch");
    cudaError_t e = cudaEventRecord(ev, d->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ns, ev, 0);
    cudaEventDestroy(ev);
    if (e != cudaSuccess) return cuda_fail(e, "stream switch");
    d->stream = ns;
  }
  return TTSH_OK;
}

ttsh_status ttsh_set_velocity(ttsh_domain* d, const double* vx, const double* vy) {
  if (!d || !vx || !vy) return fail(TTSH_E_INVALID, "NULL argument");
  const size_t NN = (size_t)d->n * d->n;
  TTSH_CUDA(cudaMemcpyAsync(d->dev.real, vx, NN * sizeof(double), cudaMemcpyHostToDevice, d->stream), "upload vx");
  TTSH_CUDA(cudaMemcpyAsync(d->dev.real + NN, vy, NN * sizeof(double), cudaMemcpyHostToDevice, d->stream), "upload vy");
  return project_staged(d);
}

ttsh_status ttsh_set_velocity_device(ttsh_domain* d, const double* vx, const double* vy) {
  if (!d || !vx || !vy) return fail(TTSH_E_INVALID, "NULL argument");
  const size_t NN = (size_t)d->n * d->n;
  TTSH_CUDA(cudaMemcpyAsync(d->dev.real, vx, NN * sizeof(double), cudaMemcpyDeviceToDevice, d->stream), "copy vx");
  TTSH_CUDA(cudaMemcpyAsync(d->dev.real + NN, vy, NN * sizeof(double), cudaMemcpyDeviceToDevice, d->stream), "copy vy");
  return project_staged(d);
}

ttsh_status ttsh_init_noise(ttsh_domain* d, uint64_t seed, double amplitude) {
  if (!d) return fail(TTSH_E_INVALID, "domain is NULL");
  if (!std::isfinite(amplitude)) return fail(TTSH_E_INVALID, "amplitude must be finite");
  const long long nn = (long long)d->n * d->n;
  const int blocks = (int)std::min<long long>((nn + 255) / 256, 152LL * 16);
  ttsh::noise_kernel<<<blocks, 256, 0, d->stream>>>(d->dev.real, d->dev.knaive, nn, (unsigned long long)seed,
                                                     amplitude);
  TTSH_CUDA(cudaGetLastError(), "noise kernel");
  return project_staged(d);
}

ttsh_status ttsh_step(ttsh_domain* d, int64_t nsteps) {
  NvtxRange nvtx_range("ttsh_step");
  if (!d) return fail(TTSH_E_INVALID, "domain is NULL");
  if (nsteps < 0) return fail(TTSH_E_INVALID, "nsteps must be >= 0");
  ttsh_status st;
  int64_t left = nsteps;
  if (left >= 2 * kGraphLen && !d->graph) {
    // one eager step first: it sets the kernels' shared-memory attributes outside capture
    if ((st = one_step(d, d->stream)) != TTSH_OK) return st;
    --left;
    d->steps += 1;
    if ((st = build_graph(d)) != TTSH_OK) return st;
  }
  if (d->graph) {
    while (left >= d->graph_len) {
      TTSH_CUDA(cudaGraphLaunch(d->graph, d->stream), "graph launch");
      left -= d->graph_len;
      d->steps += d->graph_len;
    }
  }
  for (; left > 0; --left) {
    if ((st = one_step(d, d->stream)) != TTSH_OK) return st;
    d->steps += 1;
  }
  return TTSH_OK;
}

ttsh_status ttsh_step_record(ttsh_domain* d, int64_t nsteps, int32_t every, double* series,
                             int64_t capacity, const double* centre) {
  NvtxRange nvtx_range("ttsh_step_record");
  if (!d) return fail(TTSH_E_INVALID, "domain is NULL");
  if (nsteps < 0) return fail(TTSH_E_INVALID, "nsteps must be >= 0");
  if (every < 1) return fail(TTSH_E_INVALID, "every must be >= 1");
  const int64_t nsamp = (nsteps + every - 1) / every;
  if (nsamp > 0 && !series) return fail(TTSH_E_INVALID, "series is NULL");
  if (capacity < nsamp) return fail(TTSH_E_INVALID, "capacity is smaller than the number of samples");
  if (nsamp > 0) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, series) != cudaSuccess ||
        (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
      cudaGetLastError();
      return fail(TTSH_E_INVALID, "series must be device (or managed) memory");
    }
  }
  const double cx = centre ? centre[0] : 0.0, cy = centre ? centre[1] : 0.0;
  if (!std::isfinite(cx) || !std::isfinite(cy)) return fail(TTSH_E_INVALID, "centre must be finite");
  if (d->rec_graph && (d->rec_every != every || d->rec_cx != cx || d->rec_cy != cy || d->rec_rv != d->rv ||
                       d->rec_cv != d->cv))
    drop_record_graph(d);
  d->rec_every = every;
  d->rec_cx = cx;
  d->rec_cy = cy;
  d->rec_rv = d->rv;
  d->rec_cv = d->cv;
  cudaStream_t s = d->stream;
  char* base = static_cast<char*>(d->ws);
  ttsh::record_begin_kernel<<<1, 1, 0, s>>>(reinterpret_cast<ttsh::RecCtl*>(base + d->lay.recctl), (long long)d->steps,
                                            series, capacity, every, d->n / d->ops.row_step[d->rv].rows,
                                            1.0 / (2.0 * (double)d->n * (double)d->n));
  TTSH_CUDA(cudaGetLastError(), "time-series start");
  ttsh_status st;
  int64_t i = 0;
  while (i < nsteps) {
    if (i % every == 0) {
      if (every <= kGraphLen && i > 0 && nsteps - i >= every * (kGraphLen / every)) {
        // the first sample of the call ran eagerly, so the kernels' attributes are set
        if (!d->rec_graph && (st = build_record_graph(d)) != TTSH_OK) return st;
        TTSH_CUDA(cudaGraphLaunch(d->rec_graph, s), "graph launch");
        i += d->rec_len;
        d->steps += d->rec_len;
        continue;
      }
      if ((st = record_step(d, s)) != TTSH_OK) return st;
      ++i;
      d->steps += 1;
      if (every > kGraphLen) {   // the plain steps up to the next sample
        const int64_t k = std::min<int64_t>(every - 1, nsteps - i);
        if ((st = ttsh_step(d, k)) != TTSH_OK) return st;
        i += k;
      }
      continue;
    }
    if ((st = one_step(d, s)) != TTSH_OK) return st;
    ++i;
    d->steps += 1;
  }
  return TTSH_OK;
}

ttsh_status ttsh_get_fields(ttsh_domain* d, double* vx, double* vy, double* omega) {
  if (!d) return fail(TTSH_E_INVALID, "domain is NULL");
  ttsh_status st = run_row(d, ttsh::K_ROW_INV_FIELDS, d->stream);
  if (st != TTSH_OK) return st;
  const size_t NN = (size_t)d->n * d->n;
  double* dst[3] = {omega, vx, vy};
  for (int f = 0; f < 3; ++f)
    if (dst[f])
      TTSH_CUDA(cudaMemcpyAsync(dst[f], d->dev.real + f * NN, NN * sizeof(double), cudaMemcpyDeviceToHost, d->stream),
                "download fields");
  return sync(d, "get_fields");
}

ttsh_status ttsh_get_mask(ttsh_domain* d, double* K) {
  if (!d || !K) return fail(TTSH_E_INVALID, "NULL argument");
  const size_t NN = (size_t)d->n * d->n;
  if (d->elt == sizeof(float)) {
    std::vector<float> h(NN);
    TTSH_CUDA(cudaMemcpyAsync(h.data(), d->dev.K, NN * sizeof(float), cudaMemcpyDeviceToHost, d->stream), "download K");
    if ((sync(d, "get_mask")) != TTSH_OK) return TTSH_E_CUDA;
    to_host_double(h, K);
  } else {
    TTSH_CUDA(cudaMemcpyAsync(K, d->dev.K, NN * sizeof(double), cudaMemcpyDeviceToHost, d->stream), "download K");
    return sync(d, "get_mask");
  }
  return TTSH_OK;
}

ttsh_status ttsh_get_spectral_state(ttsh_domain* d, double* w_hat, double* v0) {
  if (!d) return fail(TTSH_E_INVALID, "domain is NULL");
  const size_t ne = (size_t)d->H * d->NK * 2;
  if (d->elt == sizeof(float)) {
    std::vector<float> h(ne), m(2);
    if (w_hat) TTSH_CUDA(cudaMemcpyAsync(h.data(), d->dev.what, ne * sizeof(float), cudaMemcpyDeviceToHost, d->stream), "download state");
    TTSH_CUDA(cudaMemcpyAsync(m.data(), d->dev.vmean, 2 * sizeof(float), cudaMemcpyDeviceToHost, d->stream), "download mean");
    ttsh_status st = sync(d, "get_spectral_state");
    if (st != TTSH_OK) return st;
    if (w_hat) to_host_double(h, w_hat);
    if (v0) to_host_double(m, v0);
  } else {
    if (w_hat) TTSH_CUDA(cudaMemcpyAsync(w_hat, d->dev.what, ne * sizeof(double), cudaMemcpyDeviceToHost, d->stream), "download state");
    double m[2];
    TTSH_CUDA(cudaMemcpyAsync(m, d->dev.vmean, 2 * sizeof(double), cudaMemcpyDeviceToHost, d->stream), "download mean");
    ttsh_status st = sync(d, "get_spectral_state");
    if (st != TTSH_OK) return st;
    if (v0) {
      v0[0] = m[0];
      v0[1] = m[1];
    }
  }
  return TTSH_OK;
}

ttsh_status ttsh_set_spectral_state(ttsh_domain* d, const double* w_hat, const double* v0) {
  if (!d || !w_hat || !v0) return fail(TTSH_E_INVALID, "NULL argument");
  const size_t ne = (size_t)d->H * d->NK * 2;
  ttsh_status st;
  if (d->elt == sizeof(float)) {
    std::vector<float> h(ne), m(2);
    for (size_t i = 0; i < ne; ++i) h[i] = (float)w_hat[i];
    m[0] = (float)v0[0];
    m[1] = (float)v0[1];
    TTSH_CUDA(cudaMemcpyAsync(d->dev.what, h.data(), ne * sizeof(float), cudaMemcpyHostToDevice, d->stream), "upload state");
    TTSH_CUDA(cudaMemcpyAsync(d->dev.vmean, m.data(), 2 * sizeof(float), cudaMemcpyHostToDevice, d->stream), "upload mean");
    if ((st = sync(d, "set_spectral_state")) != TTSH_OK) return st;   // host vectors die here
  } else {
    TTSH_CUDA(cudaMemcpyAsync(d->dev.what, w_hat, ne * sizeof(double), cudaMemcpyHostToDevice, d->stream), "upload state");
    TTSH_CUDA(cudaMemcpyAsync(d->dev.vmean, v0, 2 * sizeof(double), cudaMemcpyHostToDevice, d->stream), "upload mean");
  }
  if ((st = run_col(d, ttsh::K_COL_PROLOGUE, d->stream)) != TTSH_OK) return st;
  d->steps = 0;
  return sync(d, "set_spectral_state");
}

ttsh_status ttsh_diagnostics(ttsh_domain* d, ttsh_diag* out, double* spectrum, int32_t nbins,
                             const double* centre) {
  NvtxRange nvtx_range("ttsh_diagnostics");
  if (!d || !out) return fail(TTSH_E_INVALID, "NULL argument");
  if (nbins < 0 || nbins > 65536) return fail(TTSH_E_INVALID, "nbins must be in [0, 65536]");
  if (nbins > 0 && !spectrum) return fail(TTSH_E_INVALID, "spectrum is NULL");
  d->dev.cx = centre ? centre[0] : 0.0;
  d->dev.cy = centre ? centre[1] : 0.0;
  const int nb_dev = d->M + 1;   // shells beyond N/4 hold no energy
  cudaStream_t s = d->stream;
  ttsh_status st = run_row(d, ttsh::K_ROW_INV_DIAG, s);
  if (st != TTSH_OK) return st;
  const int nblocks = d->ops.row_blocks(ttsh::K_ROW_INV_DIAG);
  TTSH_CUDA(ttsh::launch_diag_reduce(d->dev.part, nblocks, d->dev.out, s), "diag reduce");
  TTSH_CUDA(cudaMemsetAsync(d->dev.bad, 0, sizeof(int), s), "memset");
  TTSH_CUDA(d->ops.spec(d->dev, nb_dev, s), "spectrum kernel");
  const double scale = 1.0 / (2.0 * (double)d->n * (double)d->n);
  TTSH_CUDA(ttsh::launch_spectrum_reduce(d->dev.colhist, d->H, nb_dev, scale, d->dev.out + 8, s), "spectrum reduce");
  // divergence of the real-space velocity: the diagnostic row pass left DFT_x[v_x], DFT_x[v_y]
  // in the inter-pass buffer; the column pass completes the transforms and takes the maxima
  TTSH_CUDA(cudaMemsetAsync(d->dev.out + 5, 0, 2 * sizeof(double), s), "memset");
  if ((st = run_col(d, ttsh::K_COL_DIV, s)) != TTSH_OK) return st;
  std::vector<double> h(8 + nb_dev);
  int bad = 0;
  TTSH_CUDA(cudaMemcpyAsync(h.data(), d->dev.out, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s), "download diag");
  TTSH_CUDA(cudaMemcpyAsync(&bad, d->dev.bad, sizeof(int), cudaMemcpyDeviceToHost, s), "download flag");
  double vm[2];
  if (d->elt == sizeof(float)) {
    float f[2];
    TTSH_CUDA(cudaMemcpyAsync(f, d->dev.vmean, sizeof(f), cudaMemcpyDeviceToHost, s), "download mean");
    if ((st = sync(d, "diagnostics")) != TTSH_OK) return st;
    vm[0] = f[0];
    vm[1] = f[1];
  } else {
    TTSH_CUDA(cudaMemcpyAsync(vm, d->dev.vmean, sizeof(vm), cudaMemcpyDeviceToHost, s), "download mean");
    if ((st = sync(d, "diagnostics")) != TTSH_OK) return st;
  }
  const double inv2n2 = 1.0 / (2.0 * (double)d->n * (double)d->n);
  const double two_over_pi = 0.63661977236758134307553505349005744813783858296183;
  out->energy = h[0] * inv2n2;
  out->enstrophy = h[1] * inv2n2;
  out->psi = (h[2] / h[3] - two_over_pi) / (1.0 - two_over_pi);
  out->max_div = h[6] > 0.0 ? h[5] / h[6] : 0.0;
  out->mean_vx = vm[0] / d->n;
  out->mean_vy = vm[1] / d->n;
  out->step = d->steps;
  out->nonfinite = (int32_t)h[4] + bad;
  out->reserved = 0;
  for (int i = 0; i < nbins; ++i) spectrum[i] = i < nb_dev ? h[8 + i] : 0.0;
  if ((st = check_status(d)) != TTSH_OK) return st;
  if (out->nonfinite) return fail(TTSH_E_NONFINITE, "state holds non-finite values");
  return TTSH_OK;
}

ttsh_status ttsh_time_kernels(ttsh_domain* d, int32_t iters, double* ms) {
  if (!d || !ms) return fail(TTSH_E_INVALID, "NULL argument");
  if (iters < 1 || iters > 1000000) return fail(TTSH_E_INVALID, "iters must be in [1, 1000000]");
  ttsh_status st = save_state(d);
  if (st != TTSH_OK) return st;
  const int pdl = d->dev.pdl;
  d->dev.pdl = 0;   // each launch timed whole, with no overlap from the next one
  if ((st = time_launches(d, d->ops.row_step[d->rv].fn, iters, &ms[0])) == TTSH_OK)
    st = time_launches(d, d->ops.col_step[d->cv].fn, iters, &ms[1]);
  d->dev.pdl = pdl;
  if (st != TTSH_OK) return st;
  return restore_state(d);
}

ttsh_status ttsh_autotune(ttsh_domain* d, int32_t iters, int32_t* plan) {
  NvtxRange nvtx_range("ttsh_autotune");
  if (!d) return fail(TTSH_E_INVALID, "domain is NULL");
  if (iters < 1 || iters > 100000) return fail(TTSH_E_INVALID, "iters must be in [1, 100000]");
  ttsh_status st = save_state(d);
  if (st != TTSH_OK) return st;
  const int pdl0 = d->dev.pdl, tma0 = d->dev.use_tma;
  d->dev.pdl = 0;   // variants are timed as plain back-to-back launches
  double best = 1e300;
  int br = 0, bc = 0, btma = 0;
  for (int i = 0; i < d->ops.n_row_variants; ++i) {
    for (int tma = 0; tma < 1 + d->ops.row_step[i].tma; ++tma) {   // G tile by cp.async, then by TMA (where the tile allows)
      d->dev.use_tma = tma;
      double t;
      if ((st = time_launches(d, d->ops.row_step[i].fn, iters, &t)) != TTSH_OK) return st;
      if (t < best) { best = t; br = i; btma = tma; }
    }
  }
  d->dev.use_tma = btma;
  best = 1e300;
  for (int i = 0; i < d->ops.n_col_variants; ++i) {
    double t;
    if ((st = time_launches(d, d->ops.col_step[i].fn, iters, &t)) != TTSH_OK) return st;
    if (t < best) { best = t; bc = i; }
  }
  d->dev.pdl = pdl0;
  d->dev.use_tma = tma0;
  if ((st = restore_state(d)) != TTSH_OK) return st;
  if ((st = ttsh_set_plan(d, br, bc)) != TTSH_OK) return st;
  // launch mode: whole steps (row then column pass) with and without programmatic
  // dependent launch; keep the faster
  double t_mode[2];
  for (int pdl = 0; pdl < 2; ++pdl) {
    if ((st = ttsh_set_launch_mode(d, pdl | (btma << 1))) != TTSH_OK) return st;
    if ((st = save_state(d)) != TTSH_OK) return st;
    if ((st = time_steps(d, iters, &t_mode[pdl])) != TTSH_OK) return st;
    if ((st = restore_state(d)) != TTSH_OK) return st;
  }
  if ((st = ttsh_set_launch_mode(d, (t_mode[1] < t_mode[0] ? 1 : 0) | (btma << 1))) != TTSH_OK) return st;
  return ttsh_get_plan(d, plan);
}

ttsh_status ttsh_set_launch_mode(ttsh_domain* d, int32_t mode) {
  if (!d) return fail(TTSH_E_INVALID, "domain is NULL");
  if (mode < 0 || mode > 3) return fail(TTSH_E_INVALID, "launch mode must be in [0, 3]");
  const int pdl = mode & 1, tma = (mode >> 1) & 1;
  if (pdl != d->dev.pdl || tma != d->dev.use_tma) {
    if (d->graph) {
      cudaGraphExecDestroy(d->graph);
      d->graph = nullptr;
      d->graph_len = 0;
    }
    drop_record_graph(d);
    d->dev.pdl = pdl;
    d->dev.use_tma = tma;
  }
  return TTSH_OK;
}

ttsh_status ttsh_get_plan(ttsh_domain* d, int32_t* plan) {
  if (!d) return fail(TTSH_E_INVALID, "domain is NULL");
  if (plan) {
    plan[0] = d->rv;
    plan[1] = d->cv;
    plan[2] = d->ops.row_step[d->rv].rows;
    plan[3] = d->ops.row_step[d->rv].pe;
    plan[4] = d->ops.col_step[d->cv].pe;
    plan[5] = d->ops.n_row_variants;
    plan[6] = d->ops.n_col_variants;
    plan[7] = d->dev.pdl | (d->dev.use_tma << 1);
    plan[8] = d->ops.row_step[d->rv].cl;
    plan[9] = d->ops.row_step[d->rv].cmp;
  }
  return TTSH_OK;
}

ttsh_status ttsh_set_plan(ttsh_domain* d, int32_t row_variant, int32_t col_variant) {
  if (!d) return fail(TTSH_E_INVALID, "domain is NULL");
  if (row_variant < 0 || row_variant >= d->ops.n_row_variants || col_variant < 0 ||
      col_variant >= d->ops.n_col_variants)
    return fail(TTSH_E_INVALID, "variant index out of range");
  if (row_variant != d->rv || col_variant != d->cv) {
    if (d->graph) {
      cudaGraphExecDestroy(d->graph);
      d->graph = nullptr;
      d->graph_len = 0;
    }
    drop_record_graph(d);
    d->rv = row_variant;
    d->cv = col_variant;
  }
  return TTSH_OK;
}


ttsh_status ttsh_batch_create(ttsh_domain* const* domains, int32_t ndom, void* stream, ttsh_batch** out) {
  if (!out) return fail(TTSH_E_INVALID, "out is NULL");
  *out = nullptr;
  if (!domains || ndom < 1) return fail(TTSH_E_INVALID, "need at least one domain");
  std::unordered_set<ttsh_domain*> seen;
  for (int i = 0; i < ndom; ++i) {
    ttsh_domain* d = domains[i];
    if (!d) return fail(TTSH_E_INVALID, "NULL domain in batch");
    if (!seen.insert(d).second) return fail(TTSH_E_INVALID, "a domain appears twice in the batch");
    if (!d->ops.row_step[d->rv].batched || !d->ops.col_step[d->cv].batched)
      return fail(TTSH_E_UNSUPPORTED, "batched stepping supports n <= 1024");
  }
  ttsh_batch* b = new ttsh_batch();
  b->stream = static_cast<cudaStream_t>(stream);
  auto cleanup = [&](ttsh_status st) {
    ttsh_batch_destroy(b);
    return st;
  };
  for (int i = 0; i < ndom; ++i) {
    ttsh_domain* d = domains[i];
    b->all.push_back(d);
    BatchGroup* g = nullptr;
    for (auto& x : b->groups)
      if (x.precision == d->p.precision && x.n == d->n && x.rv == d->rv && x.cv == d->cv) g = &x;
    if (!g) {
      b->groups.emplace_back();
      g = &b->groups.back();
      g->precision = d->p.precision;
      g->n = d->n;
      g->rv = d->rv;
      g->cv = d->cv;
      g->row = &d->ops.row_step[d->rv];
      g->col = &d->ops.col_step[d->cv];
    }
    g->doms.push_back(d);
  }
  cudaError_t e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->order, cudaEventDisableTiming);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "batch streams"));
  // persistent mode where the batch allows it (the default then)
  {
    const int prec = b->all[0]->p.precision;
    bool ok = prec == 32 ? ttsh::persist_f32(&b->pops) : ttsh::persist_f64(&b->pops);
    for (ttsh_domain* d : b->all)
      ok = ok && d->p.precision == prec && d->n <= b->pops.max_n && b->pops.row_blocks(d->n) > 0 &&
           d->rv == 0 && d->cv == 0;
    if (ok) {
      const int nd = (int)b->all.size();
      std::vector<unsigned char> dt((size_t)b->pops.domain_bytes * nd);
      for (int k = 0; k < nd; ++k)
        b->pops.pack(b->all[k]->dev, b->pops.row_blocks(b->all[k]->n), b->all[k]->H,
                     dt.data() + (size_t)k * b->pops.domain_bytes);
      // one step's items: the domains in kGroups groups of about equal work (larger domains
      // first, each to the lightest group); the rows of every group, then the columns of
      // every group in the same order, so each item's dependencies were taken kGroups - 1
      // group-phases earlier (measured on the 48-domain sweep: two groups 66-68 us per step,
      // four groups 72 us)
      constexpr int kGroups = 2;
      std::vector<int> order(nd);
      for (int k = 0; k < nd; ++k) order[k] = k;
      std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->all[x]->n > b->all[y]->n; });
      std::vector<int> grp[kGroups];
      long long load[kGroups] = {};
      for (int k : order) {
        int w = 0;
        for (int gi = 1; gi < kGroups; ++gi)
          if (load[gi] < load[w]) w = gi;
        grp[w].push_back(k);
        load[w] += (long long)b->all[k]->n * b->all[k]->n;
      }
      std::vector<int> items;
      for (int phase = 0; phase < 2; ++phase)
        for (int gi = 0; gi < kGroups; ++gi)
          for (int k : grp[gi]) {
            const int nb = phase == 0 ? b->pops.row_blocks(b->all[k]->n) : b->all[k]->H;
            for (int blk = 0; blk < nb; ++blk) {
              items.push_back(k);
              items.push_back(phase);
              items.push_back(blk);
              items.push_back(0);
            }
          }
      b->pips = (int)(items.size() / 4);
      static_assert(sizeof(int) * 4 == 16, "work item layout");
      cudaError_t pe = b->pops.item_bytes == 16 ? cudaSuccess : cudaErrorInvalidValue;
      if (pe == cudaSuccess) pe = cudaMalloc(&b->pdoms, dt.size());
      if (pe == cudaSuccess) pe = cudaMalloc(&b->pitems, items.size() * sizeof(int));
      if (pe == cudaSuccess) pe = cudaMalloc(&b->pctl, (2 + 2 * (size_t)nd) * sizeof(unsigned long long));
      if (pe == cudaSuccess) pe = cudaMemcpy(b->pdoms, dt.data(), dt.size(), cudaMemcpyHostToDevice);
      if (pe == cudaSuccess) pe = cudaMemcpy(b->pitems, items.data(), items.size() * sizeof(int), cudaMemcpyHostToDevice);
      if (pe == cudaSuccess) pe = b->pops.prepare(&b->pgrid);
      if (pe != cudaSuccess) return cleanup(cuda_fail(pe, "persistent batch set-up"));
      b->can_persist = true;
      b->persistent = true;
    }
  }
  for (auto& g : b->groups) {
    const int ab = g.doms[0]->ops.args_bytes;
    std::vector<unsigned char> host((size_t)ab * g.doms.size());
    for (size_t k = 0; k < g.doms.size(); ++k) g.doms[k]->ops.pack_args(g.doms[k]->dev, host.data() + k * ab);
    e = cudaMalloc(&g.args_dev, host.size());
    if (e == cudaSuccess) e = cudaMemcpy(g.args_dev, host.data(), host.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g.branch, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = g.row->prepare();
    if (e == cudaSuccess) e = g.col->prepare();
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "batch set-up"));
  }
  *out = b;
  return TTSH_OK;
}

ttsh_status ttsh_batch_step(ttsh_batch* b, int64_t nsteps) {
  NvtxRange nvtx_range("ttsh_batch_step");
  if (!b) return fail(TTSH_E_INVALID, "batch is NULL");
  if (nsteps < 0) return fail(TTSH_E_INVALID, "nsteps must be >= 0");
  // work already queued on a domain's own stream comes first (a device-side wait; the host
  // does not block)
  for (ttsh_domain* d : b->all) {
    if (d->stream == b->stream) continue;
    TTSH_CUDA(cudaEventRecord(b->order, d->stream), "order event");
    TTSH_CUDA(cudaStreamWaitEvent(b->stream, b->order, 0), "order wait");
  }
  ttsh_status st;
  if (b->persistent) {
    if (nsteps > 0) {
      const size_t ctl_bytes = (2 + 2 * b->all.size()) * sizeof(unsigned long long);
      TTSH_CUDA(cudaMemsetAsync(b->pctl, 0, ctl_bytes, b->stream), "persistent batch reset");
      TTSH_CUDA(b->pops.launch(b->pdoms, b->pitems, b->pips, (long long)nsteps, b->pctl, b->pgrid, ttsh::kWaitLimitNs,
                               b->stream),
                "persistent batch launch");
    }
    for (ttsh_domain* d : b->all) d->steps += nsteps;
    return TTSH_OK;
  }
  int64_t left = nsteps;
  if (left >= kBatchGraphLen && !b->graph) {
    if ((st = batch_build_graph(b, kBatchGraphLen, &b->graph)) != TTSH_OK) return st;
    b->graph_len = kBatchGraphLen;
  }
  while (b->graph && left >= b->graph_len) {
    TTSH_CUDA(cudaGraphLaunch(b->graph, b->stream), "batch graph launch");
    left -= b->graph_len;
  }
  if (left > 0) {
    // the remainder as a graph too (cached for the next call with the same remainder, such as
    // a fixed renormalisation interval)
    if (b->tail_len != (int)left) {
      if (b->tail) cudaGraphExecDestroy(b->tail);
      b->tail = nullptr;
      b->tail_len = 0;
      if ((st = batch_build_graph(b, (int)left, &b->tail)) != TTSH_OK) return st;
      b->tail_len = (int)left;
    }
    TTSH_CUDA(cudaGraphLaunch(b->tail, b->stream), "batch graph launch");
  }
  for (ttsh_domain* d : b->all) d->steps += nsteps;
  return TTSH_OK;
}

ttsh_status ttsh_batch_synchronize(ttsh_batch* b) {
  if (!b) return fail(TTSH_E_INVALID, "batch is NULL");
  TTSH_CUDA(cudaStreamSynchronize(b->stream), "batch synchronize");
  return TTSH_OK;
}

int32_t ttsh_batch_groups(const ttsh_batch* b) { return b ? (int32_t)b->groups.size() : -1; }

ttsh_status ttsh_batch_set_persistent(ttsh_batch* b, int32_t on) {
  if (!b) return fail(TTSH_E_INVALID, "batch is NULL");
  if (on != 0 && on != 1) return fail(TTSH_E_INVALID, "on must be 0 or 1");
  if (on && !b->can_persist)
    return fail(TTSH_E_UNSUPPORTED,
                "persistent stepping needs one precision, n <= 512 and the default tile shapes in every domain");
  b->persistent = on == 1;
  return TTSH_OK;
}

int32_t ttsh_batch_persistent(const ttsh_batch* b) { return b ? (b->persistent ? 1 : 0) : -1; }

ttsh_status ttsh_batch_test_stalled_wait(ttsh_batch* b, double seconds) {
  if (!b) return fail(TTSH_E_INVALID, "batch is NULL");
  if (!(seconds > 0.0) || seconds > 1.0) return fail(TTSH_E_INVALID, "seconds must be in (0, 1]");
  if (!b->can_persist) return fail(TTSH_E_UNSUPPORTED, "the batch does not allow persistent stepping");
  // one block, one work item: the first column item of the first domain's first step, whose
  // row items are not in the list, so its dependency wait cannot complete
  if (!b->ptest) {
    const int item[4] = {0, 1, 0, 0};
    TTSH_CUDA(cudaMalloc(&b->ptest, sizeof(item)), "test item");
    TTSH_CUDA(cudaMemcpy(b->ptest, item, sizeof(item), cudaMemcpyHostToDevice), "test item");
  }
  for (ttsh_domain* d : b->all) {
    if (d->stream == b->stream) continue;
    TTSH_CUDA(cudaEventRecord(b->order, d->stream), "order event");
    TTSH_CUDA(cudaStreamWaitEvent(b->stream, b->order, 0), "order wait");
  }
  const size_t ctl_bytes = (2 + 2 * b->all.size()) * sizeof(unsigned long long);
  TTSH_CUDA(cudaMemsetAsync(b->pctl, 0, ctl_bytes, b->stream), "persistent batch reset");
  TTSH_CUDA(b->pops.launch(b->pdoms, b->ptest, 1, 1, b->pctl, 1, (unsigned long long)(seconds * 1e9), b->stream),
            "stalled persistent launch");
  return TTSH_OK;
}

void ttsh_batch_destroy(ttsh_batch* b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->tail) cudaGraphExecDestroy(b->tail);
  for (auto& g : b->groups) {
    if (g.args_dev) cudaFree(g.args_dev);
    if (g.branch) cudaStreamDestroy(g.branch);
    if (g.join) cudaEventDestroy(g.join);
  }
  if (b->pdoms) cudaFree(b->pdoms);
  if (b->ptest) cudaFree(b->ptest);
  if (b->pitems) cudaFree(b->pitems);
  if (b->pctl) cudaFree(b->pctl);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->order) cudaEventDestroy(b->order);
  if (b->capture) cudaStreamDestroy(b->capture);
  delete b;
}

ttsh_status ttsh_restrict(const ttsh_domain* fine, ttsh_domain* coarse) {
  if (!fine || !coarse) return fail(TTSH_E_INVALID, "NULL domain");
  if (fine->p.precision != coarse->p.precision) return fail(TTSH_E_INVALID, "precisions differ");
  if (coarse->n > fine->n) return fail(TTSH_E_INVALID, "coarse grid is finer than the fine grid");
  const double lf = fine->n * fine->p.dx, lc = coarse->n * coarse->p.dx;
  if (std::fabs(lf - lc) > 1e-12 * lf) return fail(TTSH_E_INVALID, "domains cover different boxes");
  TTSH_CUDA(cudaStreamSynchronize(fine->stream), "fine stream");
  const int total = coarse->H * coarse->NK;
  if (coarse->elt == sizeof(float))
    ttsh::restrict_kernel<float><<<(total + 255) / 256, 256, 0, coarse->stream>>>(
        (const ttsh::cplx<float>*)fine->dev.what, (const float*)fine->dev.vmean, fine->n,
        (ttsh::cplx<float>*)coarse->dev.what, (float*)coarse->dev.vmean, coarse->n);
  else
    ttsh::restrict_kernel<double><<<(total + 255) / 256, 256, 0, coarse->stream>>>(
        (const ttsh::cplx<double>*)fine->dev.what, (const double*)fine->dev.vmean, fine->n,
        (ttsh::cplx<double>*)coarse->dev.what, (double*)coarse->dev.vmean, coarse->n);
  TTSH_CUDA(cudaGetLastError(), "restrict kernel");
  ttsh_status st = run_col(coarse, ttsh::K_COL_PROLOGUE, coarse->stream);
  if (st != TTSH_OK) return st;
  coarse->steps = 0;
  TTSH_CUDA(cudaStreamSynchronize(coarse->stream), "restrict");
  return TTSH_OK;
}


ttsh_status ttsh_psd_begin(ttsh_domain* d, const double* omegas, int32_t nfreq) {
  if (!d || !omegas) return fail(TTSH_E_INVALID, "NULL argument");
  if (nfreq < 1 || nfreq > 4096) return fail(TTSH_E_INVALID, "nfreq must be in [1, 4096]");
  if (d->psd_omega) cudaFree(d->psd_omega);
  if (d->psd_acc) cudaFree(d->psd_acc);
  if (d->psd_S) cudaFree(d->psd_S);
  if (d->psd_S) cudaFree(d->psd_S);
  d->psd_omega = nullptr;
  d->psd_acc = nullptr;
  d->psd_S = nullptr;
  d->psd_nfreq = 0;
  const size_t nm = (size_t)d->H * d->NK;
  TTSH_CUDA(cudaMalloc(&d->psd_omega, nfreq * sizeof(double)), "PSD allocation");
  TTSH_CUDA(cudaMalloc(&d->psd_S, nfreq * sizeof(double)), "PSD allocation");
  TTSH_CUDA(cudaMalloc(&d->psd_acc, 2 * (size_t)nfreq * nm * sizeof(double2)), "PSD allocation");
  TTSH_CUDA(cudaMemcpyAsync(d->psd_omega, omegas, nfreq * sizeof(double), cudaMemcpyHostToDevice, d->stream), "PSD upload");
  TTSH_CUDA(cudaMemsetAsync(d->psd_acc, 0, 2 * (size_t)nfreq * nm * sizeof(double2), d->stream), "PSD clear");
  d->psd_nfreq = nfreq;
  return sync(d, "psd_begin");
}

ttsh_status ttsh_psd_accumulate(ttsh_domain* d, double t) {
  if (!d) return fail(TTSH_E_INVALID, "domain is NULL");
  if (!d->psd_nfreq) return fail(TTSH_E_INVALID, "ttsh_psd_begin was not called");
  const int nm = d->H * d->NK;
  dim3 grid((nm + 255) / 256, d->psd_nfreq);
  if (d->elt == sizeof(float))
    ttsh::psd_accumulate_kernel<float><<<grid, 256, 0, d->stream>>>((const ttsh::cplx<float>*)d->dev.what, nm,
                                                                    d->psd_omega, t, d->psd_acc, d->psd_nfreq);
  else
    ttsh::psd_accumulate_kernel<double><<<grid, 256, 0, d->stream>>>((const ttsh::cplx<double>*)d->dev.what, nm,
                                                                     d->psd_omega, t, d->psd_acc, d->psd_nfreq);
  TTSH_CUDA(cudaGetLastError(), "PSD accumulate");
  return TTSH_OK;
}

ttsh_status ttsh_psd_result(ttsh_domain* d, double* S) {
  if (!d || !S) return fail(TTSH_E_INVALID, "NULL argument");
  if (!d->psd_nfreq) return fail(TTSH_E_INVALID, "ttsh_psd_begin was not called");
  const double scale = 1.0 / ((double)d->n * (double)d->n);
  ttsh::psd_result_kernel<<<d->psd_nfreq, 256, 0, d->stream>>>(d->psd_acc, d->NK, d->H * d->NK, d->psd_nfreq,
                                                               scale, d->psd_S);
  TTSH_CUDA(cudaGetLastError(), "PSD result");
  std::vector<double> h(d->psd_nfreq);
  TTSH_CUDA(cudaMemcpyAsync(h.data(), d->psd_S, d->psd_nfreq * sizeof(double), cudaMemcpyDeviceToHost, d->stream),
            "PSD result");
  ttsh_status st = sync(d, "psd_result");
  if (st != TTSH_OK) return st;
  for (int j = 0; j < d->psd_nfreq; ++j) S[j] = h[j];
  return TTSH_OK;
}

ttsh_status ttsh_dumbbell_order(ttsh_domain* d, const double* centres, double radius, double* out) {
  if (!d || !centres || !out) return fail(TTSH_E_INVALID, "NULL argument");
  if (!(radius > 0)) return fail(TTSH_E_INVALID, "radius must be positive");
  ttsh_status st = run_row(d, ttsh::K_ROW_INV_FIELDS, d->stream);
  if (st != TTSH_OK) return st;
  const int nblk = 120;
  static_assert(sizeof(ttsh::Peak) * 2 * 120 <= 8192, "peak partials fit the partials region");
  ttsh::Peak* part = reinterpret_cast<ttsh::Peak*>(d->dev.part);
  ttsh::dumbbell_partial_kernel<<<nblk, 256, 0, d->stream>>>(d->dev.real, d->n, d->p.dx, centres[0], centres[1],
                                                             centres[2], centres[3], radius * radius, part);
  ttsh::dumbbell_final_kernel<<<1, 32, 0, d->stream>>>(part, nblk, d->dev.out);
  TTSH_CUDA(cudaGetLastError(), "dumbbell order");
  double h[4];
  TTSH_CUDA(cudaMemcpyAsync(h, d->dev.out, sizeof(h), cudaMemcpyDeviceToHost, d->stream), "dumbbell order");
  if ((st = sync(d, "dumbbell_order")) != TTSH_OK) return st;
  if (h[3] != 0.0) return fail(TTSH_E_INVALID, "a cavity disc contains no grid point");
  out[0] = h[0];
  out[1] = h[1];
  out[2] = h[2];
  return TTSH_OK;
}

ttsh_status ttsh_synchronize(ttsh_domain* d) {
  if (!d) return fail(TTSH_E_INVALID, "domain is NULL");
  ttsh_status st = sync(d, "synchronize");
  if (st != TTSH_OK) return st;
  return check_status(d);
}

ttsh_status ttsh_test_bounded_wait(ttsh_domain* d, double seconds) {
  if (!d) return fail(TTSH_E_INVALID, "domain is NULL");
  if (!(seconds > 0.0) || seconds > 1.0) return fail(TTSH_E_INVALID, "seconds must be in (0, 1]");
  ttsh::expire_wait_kernel<<<1, 32, 0, d->stream>>>(d->dev.err, (unsigned long long)(seconds * 1e9));
  TTSH_CUDA(cudaGetLastError(), "bounded-wait test launch");
  return TTSH_OK;
}

int64_t ttsh_step_count(const ttsh_domain* d) { return d ? d->steps : -1; }

const char* ttsh_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
