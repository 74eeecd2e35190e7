// ttsh_lyap.cu - Lyapunov exponents of a domain's trajectory (Sec. III.C: the growth rates of
// independent perturbations evolved along with the solution, obtained from QR
// decompositions by the standard method of Shimada & Nagashima (1979) and Benettin et al.
// (1980)).
//
// The k perturbations are k copies of the domain (same mask, parameters, plan and stream),
// stepped with it as one batched launch group.  After every `interval` steps each copy's
// difference from the base state, divided by eps, is the evolved perturbation (a finite
// difference of the scheme of Algorithm 1); the k differences are re-orthonormalised by
// classical Gram-Schmidt applied twice (CGS2, which reaches the orthogonality of a
// Householder QR) and the copies are reset to base + eps q_i.  log R_ii is accumulated; the
// exponents are the sums divided by the elapsed time.
//
// State vectors (length D = 2 H NK + 2 doubles) are the stored half spectrum of omega^
// (interleaved re/im, columns mx = 0..N/4) followed by v^(0); the inner product weights the
// mx > 0 columns by 2 (they stand for +-mx) so that it equals sum_x omega omega' + v^(0).v'^(0)
// (Parseval).  All reductions are block partial sums in a fixed order (repeatable bits).
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "ttsh.h"
#include "ttsh_ops.h"

namespace lyap_dev {

constexpr int kMaxK = 16;
constexpr int kBlocks = 120;   // partial-sum blocks of the dot products
constexpr int kThreads = 256;

__device__ __forceinline__ double weight(long long x, long long col2, long long D) {
  return (x < col2 || x >= D - 2) ? 1.0 : 2.0;   // mx = 0 column and mean: 1; mx > 0: 2
}

// Dl[i][x] = (pert_i[x] - base[x]) * inv_eps for i < k (pointer table: [0] base, [1..k])
template <typename T>
__global__ void diff_kernel(const T* const* __restrict__ what, const T* const* __restrict__ vmean, int k,
                            long long D, double inv_eps, double* __restrict__ Dl) {
  const int i = blockIdx.y;
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < D; x += (long long)gridDim.x * blockDim.x) {
    double a, b;
    if (x < D - 2) {
      a = (double)what[1 + i][x];
      b = (double)what[0][x];
    } else {
      a = (double)vmean[1 + i][x - (D - 2)];
      b = (double)vmean[0][x - (D - 2)];
    }
    Dl[(size_t)i * D + x] = (a - b) * inv_eps;
  }
}

// Block partials of <v, Q_j> for j < nq and, with self, <v, v> in slot nq.
__global__ void dots_kernel(const double* __restrict__ v, const double* __restrict__ Q, int nq, int self,
                            long long D, long long col2, double* __restrict__ partial) {
  __shared__ double red[kThreads];
  double acc[kMaxK + 1];
  const int nd = nq + (self ? 1 : 0);
  for (int j = 0; j < nd; ++j) acc[j] = 0.0;
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < D; x += (long long)gridDim.x * blockDim.x) {
    const double wv = weight(x, col2, D) * v[x];
    for (int j = 0; j < nq; ++j) acc[j] += wv * Q[(size_t)j * D + x];
    if (self) acc[nq] += wv * v[x];
  }
  for (int j = 0; j < nd; ++j) {
    red[threadIdx.x] = acc[j];
    __syncthreads();
    for (int s = kThreads / 2; s >= 1; s >>= 1) {
      if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) partial[(size_t)blockIdx.x * (kMaxK + 1) + j] = red[0];
    __syncthreads();
  }
}

// Slot j of the block partials summed over the nb blocks in block order (every consumer
// block computes the same sum, so no separate reduction launch is needed).
__device__ __forceinline__ double partial_sum(const double* __restrict__ partial, int nb, int j) {
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += partial[(size_t)b * (kMaxK + 1) + j];
  return s;
}

// v -= sum_j c_j Q_j (j in order), c_j = <v, Q_j> from the partials of slots 0..nq-1.  With
// norm, the block partial of <v, v> of the result goes to slot kMaxK (same summation order
// as dots_kernel with self).
__global__ void axpy_kernel(double* __restrict__ v, const double* __restrict__ Q, double* __restrict__ partial,
                            int nb, int nq, long long D, long long col2, int norm) {
  __shared__ double c[kMaxK];
  __shared__ double red[kThreads];
  if ((int)threadIdx.x < nq) c[threadIdx.x] = partial_sum(partial, nb, threadIdx.x);
  __syncthreads();
  double acc = 0.0;
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < D; x += (long long)gridDim.x * blockDim.x) {
    double s = v[x];
    for (int j = 0; j < nq; ++j) s -= c[j] * Q[(size_t)j * D + x];
    v[x] = s;
    if (norm) {
      const double wv = weight(x, col2, D) * s;
      acc += wv * s;
    }
  }
  if (norm) {
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int t = kThreads / 2; t >= 1; t >>= 1) {
      if ((int)threadIdx.x < t) red[threadIdx.x] += red[threadIdx.x + t];
      __syncthreads();
    }
    if (threadIdx.x == 0) partial[(size_t)blockIdx.x * (kMaxK + 1) + kMaxK] = red[0];
  }
}

// q = v / r with r = sqrt(<v, v>) from the partials of `slot`; with accumulate,
// logs[i] += log r and last[i] = log r.
__global__ void scale_kernel(const double* __restrict__ v, double* __restrict__ q, const double* __restrict__ partial,
                             int nb, int slot, long long D, int i, int accumulate, double* __restrict__ logs,
                             double* __restrict__ last) {
  __shared__ double r2;
  if (threadIdx.x == 0) r2 = partial_sum(partial, nb, slot);
  __syncthreads();
  const double r = sqrt(r2);
  const double inv = 1.0 / r;
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < D; x += (long long)gridDim.x * blockDim.x)
    q[x] = v[x] * inv;
  if (accumulate && blockIdx.x == 0 && threadIdx.x == 0) {
    const double l = log(r);
    logs[i] += l;
    last[i] = l;
  }
}

// pert_i = base + eps Q_i, rounded to the domain precision
template <typename T>
__global__ void set_kernel(T* const* __restrict__ what, T* const* __restrict__ vmean, const double* __restrict__ Q,
                           long long D, double eps) {
  const int i = blockIdx.y;
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < D; x += (long long)gridDim.x * blockDim.x) {
    const double q = Q[(size_t)i * D + x];
    if (x < D - 2) what[1 + i][x] = (T)((double)what[0][x] + eps * q);
    else vmean[1 + i][x - (D - 2)] = (T)((double)vmean[0][x - (D - 2)] + eps * q);
  }
}

__global__ void finish_kernel(const double* __restrict__ logs, const double* __restrict__ last, int k,
                              double inv_time, double inv_interval_time, double* __restrict__ out) {
  const int i = threadIdx.x;
  if (i >= k) return;
  out[i] = logs[i] * inv_time;
  out[k + i] = last[i] * inv_interval_time;
}

}  // namespace lyap_dev

struct ttsh_lyap {
  ttsh_domain* base = nullptr;
  std::vector<ttsh_domain*> perts;
  ttsh_batch* batch = nullptr;
  cudaStream_t stream = nullptr;
  int k = 0, precision = 32;
  long long D = 0, col2 = 0;
  double eps = 0.0, dt = 0.0;
  double* Q = nullptr;       // [k][D] orthonormal directions
  double* Dl = nullptr;      // [k][D] evolved perturbations
  double* partial = nullptr; // [kBlocks][kMaxK + 1]: dot-product partials; slot kMaxK: norms
  double* logs = nullptr;    // [k]
  double* last = nullptr;    // [k]
  double* out = nullptr;     // [2k]
  void** ptrs = nullptr;     // [2][k + 1]: what pointers, vmean pointers
  long long steps = 0, intervals = 0;
  int interval = 0;
  cudaStream_t cap = nullptr;          // private stream the renormalisation graph is captured on
  cudaGraphExec_t renorm = nullptr;    // differences + CGS2 + reset of the copies, replayed per interval
};

namespace {

ttsh_status lfail(ttsh_status s, const char* msg) {
  ttsh::set_last_error(msg);
  return s;
}

#define LY_CUDA(expr, what)                          \
  do {                                               \
    cudaError_t e_ = (expr);                         \
    if (e_ != cudaSuccess) {                         \
      ttsh::set_last_error(what, e_);                \
      return TTSH_E_CUDA;                            \
    }                                                \
  } while (0)

int grid_for(long long D) {
  long long g = (D + lyap_dev::kThreads - 1) / lyap_dev::kThreads;
  return (int)(g < lyap_dev::kBlocks ? g : lyap_dev::kBlocks);
}

// Orthonormalise the k rows of L->Dl into L->Q (CGS2); with accumulate, record log R_ii.
ttsh_status orthonormalise(ttsh_lyap* L, bool accumulate, cudaStream_t s) {
  using namespace lyap_dev;
  const int nb = grid_for(L->D);
  // per vector: two projection passes (dots, then axpy reducing the dots' partials itself;
  // the second axpy also forms the norm's partials), then the scaling
  for (int i = 0; i < L->k; ++i) {
    double* v = L->Dl + (size_t)i * L->D;
    int slot = 0;
    if (i > 0) {
      for (int pass = 0; pass < 2; ++pass) {
        dots_kernel<<<nb, kThreads, 0, s>>>(v, L->Q, i, 0, L->D, L->col2, L->partial);
        axpy_kernel<<<nb, kThreads, 0, s>>>(v, L->Q, L->partial, nb, i, L->D, L->col2, pass);
      }
      slot = kMaxK;
    } else {
      dots_kernel<<<nb, kThreads, 0, s>>>(v, L->Q, 0, 1, L->D, L->col2, L->partial);
    }
    scale_kernel<<<nb, kThreads, 0, s>>>(v, L->Q + (size_t)i * L->D, L->partial, nb, slot, L->D, i,
                                         accumulate ? 1 : 0, L->logs, L->last);
  }
  LY_CUDA(cudaGetLastError(), "orthonormalisation launch");
  return TTSH_OK;
}

// Reset every copy to base + eps Q_i and rebuild its inter-pass buffers.
ttsh_status reset_copies(ttsh_lyap* L, cudaStream_t s) {
  dim3 g(grid_for(L->D), L->k);
  void** w = L->ptrs;
  void** m = L->ptrs + (L->k + 1);
  if (L->precision == 32)
    lyap_dev::set_kernel<float><<<g, lyap_dev::kThreads, 0, s>>>(
        reinterpret_cast<float* const*>(w), reinterpret_cast<float* const*>(m), L->Q, L->D, L->eps);
  else
    lyap_dev::set_kernel<double><<<g, lyap_dev::kThreads, 0, s>>>(
        reinterpret_cast<double* const*>(w), reinterpret_cast<double* const*>(m), L->Q, L->D, L->eps);
  LY_CUDA(cudaGetLastError(), "perturbation reset launch");
  for (ttsh_domain* p : L->perts) {
    const int st = ttsh::domain_refresh_on(p, s);
    if (st != TTSH_OK) return (ttsh_status)st;
  }
  return TTSH_OK;
}

ttsh_status differences(ttsh_lyap* L, cudaStream_t s) {
  dim3 g(grid_for(L->D), L->k);
  void** w = L->ptrs;
  void** m = L->ptrs + (L->k + 1);
  if (L->precision == 32)
    lyap_dev::diff_kernel<float><<<g, lyap_dev::kThreads, 0, s>>>(
        reinterpret_cast<const float* const*>(w), reinterpret_cast<const float* const*>(m), L->k, L->D,
        1.0 / L->eps, L->Dl);
  else
    lyap_dev::diff_kernel<double><<<g, lyap_dev::kThreads, 0, s>>>(
        reinterpret_cast<const double* const*>(w), reinterpret_cast<const double* const*>(m), L->k, L->D,
        1.0 / L->eps, L->Dl);
  LY_CUDA(cudaGetLastError(), "difference launch");
  return TTSH_OK;
}

// The end-of-interval work (differences, CGS2 with accumulation, reset of the copies) is the
// same launch sequence with the same arguments every interval: capture it once on a private
// stream and replay it on the domains' stream.
ttsh_status renormalise(ttsh_lyap* L) {
  if (!L->renorm) {
    if (!L->cap) LY_CUDA(cudaStreamCreateWithFlags(&L->cap, cudaStreamNonBlocking), "capture stream");
    LY_CUDA(cudaStreamBeginCapture(L->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    ttsh_status st = differences(L, L->cap);
    if (st == TTSH_OK) st = orthonormalise(L, true, L->cap);
    if (st == TTSH_OK) st = reset_copies(L, L->cap);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(L->cap, &g);
    if (st != TTSH_OK || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      if (st != TTSH_OK) return st;
      LY_CUDA(e, "renormalisation capture");
    }
    const cudaError_t ei = cudaGraphInstantiate(&L->renorm, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      L->renorm = nullptr;
      LY_CUDA(ei, "renormalisation graph");
    }
  }
  LY_CUDA(cudaGraphLaunch(L->renorm, L->stream), "renormalisation replay");
  return TTSH_OK;
}

}  // namespace

extern "C" {

void ttsh_lyap_destroy(ttsh_lyap* L) {
  if (!L) return;
  if (L->renorm) cudaGraphExecDestroy(L->renorm);
  if (L->cap) cudaStreamDestroy(L->cap);
  if (L->batch) ttsh_batch_destroy(L->batch);
  for (ttsh_domain* p : L->perts) ttsh_destroy_domain(p);
  for (void* q : {(void*)L->Q, (void*)L->Dl, (void*)L->partial, (void*)L->logs, (void*)L->last,
                  (void*)L->out, (void*)L->ptrs})
    if (q) cudaFree(q);
  delete L;
}

ttsh_status ttsh_lyap_create(ttsh_domain* base, int32_t k, double eps, const double* q0, ttsh_lyap** out) {
  if (!out) return lfail(TTSH_E_INVALID, "out is NULL");
  *out = nullptr;
  if (!base || !q0) return lfail(TTSH_E_INVALID, "NULL argument");
  if (k < 1 || k > lyap_dev::kMaxK) return lfail(TTSH_E_INVALID, "k must be in [1, 16]");
  if (!(eps > 0) || !std::isfinite(eps)) return lfail(TTSH_E_INVALID, "eps must be positive and finite");
  ttsh_lyap* L = new ttsh_lyap();
  auto cleanup = [&](ttsh_status st) {
    ttsh_lyap_destroy(L);
    return st;
  };
  const int n = ttsh::domain_n(base);
  const long long H = n / 4 + 1, NK = n / 2 + 1;
  L->base = base;
  L->k = k;
  L->eps = eps;
  L->dt = ttsh::domain_dt(base);
  L->precision = ttsh::domain_precision(base);
  L->stream = ttsh::domain_stream(base);
  L->D = 2 * H * NK + 2;
  L->col2 = 2 * NK;
  for (int i = 0; i < k; ++i) {
    ttsh_domain* c = nullptr;
    const int st = ttsh::domain_clone(base, &c);
    if (st != TTSH_OK) return cleanup((ttsh_status)st);
    L->perts.push_back(c);
  }
  const size_t kd = (size_t)k * L->D * sizeof(double);
  cudaError_t e = cudaMalloc(&L->Q, kd);
  if (e == cudaSuccess) e = cudaMalloc(&L->Dl, kd);
  if (e == cudaSuccess) e = cudaMalloc(&L->partial, (size_t)lyap_dev::kBlocks * (lyap_dev::kMaxK + 1) * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&L->logs, k * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&L->last, k * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&L->out, 2 * k * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&L->ptrs, 2 * (k + 1) * sizeof(void*));
  if (e != cudaSuccess) {
    ttsh::set_last_error("Lyapunov buffers", e);
    return cleanup(e == cudaErrorMemoryAllocation ? TTSH_E_OOM : TTSH_E_CUDA);
  }
  std::vector<void*> hp(2 * (k + 1));
  hp[0] = ttsh::domain_dev(base)->what;
  hp[k + 1] = ttsh::domain_dev(base)->vmean;
  for (int i = 0; i < k; ++i) {
    hp[1 + i] = ttsh::domain_dev(L->perts[i])->what;
    hp[k + 2 + i] = ttsh::domain_dev(L->perts[i])->vmean;
  }
  cudaStream_t s = L->stream;
  e = cudaMemcpyAsync(L->ptrs, hp.data(), hp.size() * sizeof(void*), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(L->Dl, q0, kd, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(L->logs, 0, k * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(L->last, 0, k * sizeof(double), s);
  if (e != cudaSuccess) {
    ttsh::set_last_error("Lyapunov set-up copies", e);
    return cleanup(TTSH_E_CUDA);
  }
  ttsh_status st = orthonormalise(L, false, s);
  if (st == TTSH_OK) st = reset_copies(L, s);
  if (st != TTSH_OK) return cleanup(st);
  // batched stepping of the base and its copies where the grid allows it
  std::vector<ttsh_domain*> all{base};
  all.insert(all.end(), L->perts.begin(), L->perts.end());
  ttsh_batch* b = nullptr;
  if (n <= 1024) {
    st = ttsh_batch_create(all.data(), (int32_t)all.size(), s, &b);
    if (st != TTSH_OK) return cleanup(st);
    L->batch = b;
  }
  e = cudaStreamSynchronize(s);   // the host pointer table and q0 are read before returning
  if (e != cudaSuccess) {
    ttsh::set_last_error("Lyapunov set-up", e);
    return cleanup(TTSH_E_CUDA);
  }
  *out = L;
  return TTSH_OK;
}

ttsh_status ttsh_lyap_step(ttsh_lyap* L, int64_t nsteps, int32_t interval) {
  if (!L) return lfail(TTSH_E_INVALID, "handle is NULL");
  if (interval < 1) return lfail(TTSH_E_INVALID, "interval must be >= 1");
  if (nsteps < 0 || nsteps % interval) return lfail(TTSH_E_INVALID, "nsteps must be a non-negative multiple of interval");
  if (L->interval && L->interval != interval)
    return lfail(TTSH_E_INVALID, "interval must stay the same over a run");
  L->interval = interval;
  ttsh_status st;
  for (int64_t done = 0; done < nsteps; done += interval) {
    if (L->batch) {
      if ((st = ttsh_batch_step(L->batch, interval)) != TTSH_OK) return st;
    } else {
      if ((st = ttsh_step(L->base, interval)) != TTSH_OK) return st;
      for (ttsh_domain* p : L->perts)
        if ((st = ttsh_step(p, interval)) != TTSH_OK) return st;
    }
    if ((st = renormalise(L)) != TTSH_OK) return st;
    L->steps += interval;
    L->intervals += 1;
  }
  return TTSH_OK;
}

ttsh_status ttsh_lyap_result(ttsh_lyap* L, double* exponents, double* last_rates) {
  if (!L || !exponents) return lfail(TTSH_E_INVALID, "NULL argument");
  if (L->intervals == 0) return lfail(TTSH_E_INVALID, "no interval has been completed");
  const double T = (double)L->steps * L->dt;
  lyap_dev::finish_kernel<<<1, 32, 0, L->stream>>>(L->logs, L->last, L->k, 1.0 / T, 1.0 / (L->interval * L->dt), L->out);
  LY_CUDA(cudaGetLastError(), "Lyapunov result launch");
  std::vector<double> h(2 * L->k);
  LY_CUDA(cudaMemcpyAsync(h.data(), L->out, h.size() * sizeof(double), cudaMemcpyDeviceToHost, L->stream), "download");
  LY_CUDA(cudaStreamSynchronize(L->stream), "Lyapunov result");
  for (int i = 0; i < L->k; ++i) {
    exponents[i] = h[i];
    if (last_rates) last_rates[i] = h[L->k + i];
  }
  return TTSH_OK;
}

ttsh_status ttsh_lyap_directions(ttsh_lyap* L, double* q) {
  if (!L || !q) return lfail(TTSH_E_INVALID, "NULL argument");
  LY_CUDA(cudaMemcpyAsync(q, L->Q, (size_t)L->k * L->D * sizeof(double), cudaMemcpyDeviceToHost, L->stream), "download");
  LY_CUDA(cudaStreamSynchronize(L->stream), "Lyapunov directions");
  return TTSH_OK;
}

}  // extern "C"
