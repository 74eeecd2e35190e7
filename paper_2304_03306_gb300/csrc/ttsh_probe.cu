// ttsh_probe.cu - measured arithmetic peak of this GPU for the roofline of the ALU-bound
// (double precision) solver path: ttsh_fma_peak.
//
// Every thread runs kChains independent fused multiply-add chains x <- x * a + b for `iters`
// iterations (no memory traffic inside the loop, enough chains per thread to cover the FMA
// pipeline's latency), on a grid of several resident blocks per SM.  The rate is
// 2 flops x chains x iterations x threads / the kernel time from CUDA events.
#include <cuda_runtime.h>

#include <cmath>

#include "ttsh.h"
#include "ttsh_ops.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_probe_kernel(int iters, T a, T b, T* sink) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == (T)-1.2345) sink[0] = s;   // keeps the chains live; never true for these inputs
}

template <typename T>
ttsh_status run_probe(int iters, double* tflops) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    ttsh::set_last_error("device query", e);
    return TTSH_E_CUDA;
  }
  const int blocks = sms * 8;   // 8 blocks of 256 threads per SM: 64 warps, full occupancy
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  T* sink = nullptr;   // never written (see the kernel); a valid address all the same
  e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&sink), sizeof(T), s);
  const T a = (T)0.999999, b = (T)1e-6;   // |x| stays bounded: x -> b / (1 - a)
  float ms = 0.f;
  if (e == cudaSuccess) {
    fma_probe_kernel<T><<<blocks, kThreads, 0, s>>>(iters / 8 + 1, a, b, sink);   // warm-up
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) {
    fma_probe_kernel<T><<<blocks, kThreads, 0, s>>>(iters, a, b, sink);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (sink) cudaFreeAsync(sink, s);
  if (s) cudaStreamSynchronize(s);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (e != cudaSuccess) {
    ttsh::set_last_error("FMA probe", e);
    return TTSH_E_CUDA;
  }
  const double flops = 2.0 * kChains * (double)iters * (double)blocks * kThreads;
  *tflops = flops / ((double)ms * 1e-3) / 1e12;
  return TTSH_OK;
}

}  // namespace

extern "C" ttsh_status ttsh_fma_peak(int32_t precision, int32_t iters, double* tflops) {
  if (!tflops) {
    ttsh::set_last_error("tflops is NULL");
    return TTSH_E_INVALID;
  }
  if (iters < 1 || iters > (1 << 24)) {
    ttsh::set_last_error("iters must be in [1, 2^24]");
    return TTSH_E_INVALID;
  }
  if (precision == 32) return run_probe<float>(iters, tflops);
  if (precision == 64) return run_probe<double>(iters, tflops);
  ttsh::set_last_error("precision must be 32 or 64");
  return TTSH_E_INVALID;
}
