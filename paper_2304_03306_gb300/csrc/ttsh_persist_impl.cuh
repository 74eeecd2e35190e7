// ttsh_persist_impl.cuh - host side of the persistent batched stepper for one precision;
// included by ttsh_persist_f32.cu / ttsh_persist_f64.cu, which define TTSH_T and
// TTSH_PERSIST_REGISTRY.
#pragma once

#include <atomic>
#include <cstring>

#include "ttsh_args.cuh"
#include "ttsh_persist.cuh"

namespace ttsh {

template <typename T>
static void persist_pack(const DomainDev& d, int nrow, int ncol, void* dst) {
  PDomain<T> p;
  memset(&p, 0, sizeof(p));
  p.A = make_args<T>(d);
  p.A.aux = nullptr;
  p.n = d.n;
  p.nrow = nrow;
  p.ncol = ncol;
  memcpy(dst, &p, sizeof(p));
}

template <typename T>
static int persist_rows(int n) {
  switch (n) {
    case 16: return 16 / PersistShape<T, 16>::R;
    case 32: return 32 / PersistShape<T, 32>::R;
    case 64: return 64 / PersistShape<T, 64>::R;
    case 128: return 128 / PersistShape<T, 128>::R;
    case 256: return 256 / PersistShape<T, 256>::R;
    case 512: return 512 / PersistShape<T, 512>::R;
  }
  return 0;
}

template <typename T>
static cudaError_t persist_prepare(int* grid) {
  static std::atomic<int> cached{0};
  const int c = cached.load(std::memory_order_acquire);
  if (c > 0) {
    *grid = c;
    return cudaSuccess;
  }
  constexpr int smem = PersistLimits<T>::SMEM + 128;
  cudaError_t e = cudaFuncSetAttribute(persistent_step_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  int dev = 0, sms = 0, per_sm = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_step_kernel<T>, PersistLimits<T>::NT + 32,
                                                      smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  *grid = sms * per_sm;
  cached.store(*grid, std::memory_order_release);
  return cudaSuccess;
}

template <typename T>
static cudaError_t persist_launch(const void* doms, const void* items, int ips, long long nsteps,
                                  unsigned long long* ctl, int grid, unsigned long long limit_ns, cudaStream_t s) {
  constexpr int smem = PersistLimits<T>::SMEM + 128;
  persistent_step_kernel<T><<<grid, PersistLimits<T>::NT + 32, smem, s>>>(
      static_cast<const PDomain<T>*>(doms), static_cast<const PItem*>(items), ips, nsteps, ctl, limit_ns);
  return cudaGetLastError();
}

bool TTSH_PERSIST_REGISTRY(PersistOps* o) {
  o->launch = &persist_launch<TTSH_T>;
  o->prepare = &persist_prepare<TTSH_T>;
  o->pack = &persist_pack<TTSH_T>;
  o->row_blocks = &persist_rows<TTSH_T>;
  o->domain_bytes = (int)sizeof(PDomain<TTSH_T>);
  o->item_bytes = (int)sizeof(PItem);
  o->max_n = kPersistMaxN;
  o->threads = PersistLimits<TTSH_T>::NT + 32;
  return true;
}

}  // namespace ttsh
