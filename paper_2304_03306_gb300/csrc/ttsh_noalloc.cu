// ttsh_noalloc.cu - ttsh_step_noalloc: advance a caller-owned spectral state without any
// device allocation.
//
// Who needs this: callers whose device memory is owned by their own allocator or budget
// (a framework's caching pool, a fixed-size arena on a shared GPU, a latency-critical loop
// that must not stall on the implicit device synchronisation of cudaMalloc/cudaFree) cannot
// let a library allocate behind their back, and ttsh_create_domain allocates its workspace
// unless one is handed in.  This entry point takes the state, mask and mean flow as the
// caller's device buffers and keeps its only scratch - the two inter-pass buffers of the
// row/column step and the twiddle tables - in one file-scope device array of fixed size.
//
// The array is sized for grids up to kNoAllocMaxN = 512 in double precision (about 6.4 MB);
// every GPU that loads the library holds it until the process exits.  All calls share it:
// calls that overlap on the GPU (different streams, or different host threads, at the same
// time) race on it and must be serialised by the caller.  Nothing in it has to start at
// zero: each call first rebuilds the whole inverse-transformed buffer from the caller's
// state, and every element a pass reads was written earlier in the same call; the twiddle
// tables are written once per device, and that first call waits until they are on the
// device.
//
// Every wait inside the kernels is bounded (the column pass's bulk-copy completion), but
// this entry point has no status word to report a wait that ran out: the domain path
// reports it as TTSH_E_TIMEOUT at its next synchronising call, here the step simply goes on
// (the state of that call is then not valid).  No such wait has ever run out; callers that
// need the report use the domain path.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "ttsh.h"
#include "ttsh_ops.h"

namespace {

constexpr int kNoAllocMaxN = 512;
constexpr size_t kMaxH = kNoAllocMaxN / 4 + 1;
constexpr size_t kGBytes = 3 * kMaxH * kNoAllocMaxN * 2 * sizeof(double);
constexpr size_t kRBytes = 3 * kMaxH * kNoAllocMaxN * 2 * sizeof(double);
// twiddle tables for n = 16, 32, ..., 512: table n starts at entry n - 16
constexpr size_t kTwEntries = 2 * kNoAllocMaxN - 16;
constexpr size_t kTwF32Bytes = kTwEntries * 2 * sizeof(float);
constexpr size_t kTwF64Bytes = kTwEntries * 2 * sizeof(double);
constexpr size_t kTwF32Off = kGBytes + kRBytes;
constexpr size_t kTwF64Off = kTwF32Off + ((kTwF32Bytes + 255) / 256) * 256;
constexpr size_t kScratchBytes = kTwF64Off + kTwF64Bytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
char* g_scratch_ptr[kMaxDevices] = {};
// host images of the twiddle tables (static storage: no heap allocation)
double g_tw_host_f64[2 * kTwEntries];
float g_tw_host_f32[2 * kTwEntries];

ttsh_status bad(ttsh_status s, const char* msg) {
  ttsh::set_last_error(msg);
  return s;
}

ttsh_status cuda_bad(cudaError_t e, const char* what) {
  ttsh::set_last_error(what, e);
  return TTSH_E_CUDA;
}

// Once per device, with that device current: resolve the array's device address and write
// the twiddle tables W_n^m = exp(-2 pi i m / n) (extended precision, rounded once).
ttsh_status setup_device(int dev, char** out) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (g_scratch_ptr[dev]) {
    *out = g_scratch_ptr[dev];
    return TTSH_OK;
  }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) return cuda_bad(e, "cudaGetSymbolAddress(no-allocation scratch)");
  const long double two_pi = 6.283185307179586476925286766559005768L;
  for (int n = 16; n <= kNoAllocMaxN; n *= 2) {
    const size_t off = (size_t)(n - 16);
    for (int m = 0; m < n; ++m) {
      const long double ang = two_pi * (long double)m / (long double)n;
      const double c = (double)cosl(ang), s = (double)(-sinl(ang));
      g_tw_host_f64[2 * (off + m)] = c;
      g_tw_host_f64[2 * (off + m) + 1] = s;
      g_tw_host_f32[2 * (off + m)] = (float)c;
      g_tw_host_f32[2 * (off + m) + 1] = (float)s;
    }
  }
  char* base = static_cast<char*>(p);
  e = cudaMemcpy(base + kTwF32Off, g_tw_host_f32, kTwF32Bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(base + kTwF64Off, g_tw_host_f64, kTwF64Bytes, cudaMemcpyHostToDevice);
  // A copy from pageable host memory may return before it has reached the device, and a
  // non-blocking caller stream does not wait for the legacy stream the copies ran on: wait
  // for them here, before any kernel on the caller's stream can read the tables.
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_bad(e, "twiddle upload to the no-allocation scratch");
  g_scratch_ptr[dev] = base;
  *out = base;
  return TTSH_OK;
}

}  // namespace

extern "C" ttsh_status ttsh_step_noalloc(const ttsh_params* p, const void* K, void* w_hat, void* v0,
                                         int64_t nsteps, void* stream) {
  if (!p || !K || !w_hat || !v0) return bad(TTSH_E_INVALID, "NULL argument");
  if (p->n < 16 || (p->n & (p->n - 1)) != 0)
    return bad(TTSH_E_INVALID, "n must be a power of two >= 16");
  if (p->n > kNoAllocMaxN)
    return bad(TTSH_E_INVALID, "n exceeds the no-allocation scratch limit of 512");
  if (p->precision != 32 && p->precision != 64) return bad(TTSH_E_INVALID, "precision must be 32 or 64");
  if (!(p->dx > 0) || !(p->dt > 0) || !std::isfinite(p->dx) || !std::isfinite(p->dt))
    return bad(TTSH_E_INVALID, "dx and dt must be positive and finite");
  const double c[5] = {p->a, p->b, p->lambda, p->gamma_v, p->gamma_w};
  for (double v : c)
    if (!std::isfinite(v)) return bad(TTSH_E_INVALID, "model coefficients must be finite");
  if (nsteps < 0) return bad(TTSH_E_INVALID, "nsteps must be >= 0");
  // the kernels stage K and w_hat with 16-byte copies and read complex values as pairs
  if ((reinterpret_cast<uintptr_t>(K) | reinterpret_cast<uintptr_t>(w_hat) | reinterpret_cast<uintptr_t>(v0)) % 16 != 0)
    return bad(TTSH_E_INVALID, "K, w_hat and v0 must be 16-byte aligned");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_bad(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return bad(TTSH_E_UNSUPPORTED, "device index beyond 63");
  char* base = nullptr;
  ttsh_status st = setup_device(dev, &base);
  if (st != TTSH_OK) return st;

  ttsh::SizeOps ops;
  const bool found = p->precision == 32 ? ttsh::ops_f32_small(p->n, &ops) : ttsh::ops_f64_small(p->n, &ops);
  if (!found) return bad(TTSH_E_UNSUPPORTED, "no kernels for this grid size");

  ttsh::DomainDev d{};
  d.what = w_hat;
  d.vmean = v0;
  d.K = const_cast<void*>(K);
  d.G = base;
  d.Rr = base + kGBytes;
  d.tw = base + (p->precision == 32 ? kTwF32Off + (size_t)(p->n - 16) * 2 * sizeof(float)
                                    : kTwF64Off + (size_t)(p->n - 16) * 2 * sizeof(double));
  d.a = p->a;
  d.b = p->b;
  d.lam = p->lambda;
  d.gv = p->gamma_v;
  d.gw = p->gamma_w;
  d.dx = p->dx;
  d.dt = p->dt;
  d.n = p->n;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // rebuild the row-pass inputs from the caller's state, then step
  e = ops.col(ttsh::K_COL_PROLOGUE, d, s);
  for (int64_t i = 0; i < nsteps && e == cudaSuccess; ++i) {
    e = ops.row(ttsh::K_ROW_STEP, d, s);
    if (e == cudaSuccess) e = ops.col(ttsh::K_COL_STEP, d, s);
  }
  if (e != cudaSuccess) return cuda_bad(e, "kernel launch");
  return TTSH_OK;
}
