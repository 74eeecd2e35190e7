// ttsh_persist.cuh - persistent batched stepper: one launch advances a batch of independent
// domains of uneven grid sizes (the paper's radius and dumbbell sweeps, Sec. III.C and
// Sec. IV) by any number of steps.
//
// Work items.  Step s of domain d is its row pass (nrow blocks of work) followed by its
// column pass (ncol blocks of work), exactly the blocks the single-domain kernels launch.
// Every (step, domain, pass, block) is one item; the items of one step are listed once and
// the launch walks the list nsteps times: item g is list entry g mod (items per step) of
// step g / (items per step).  Resident blocks take items in increasing g from one global
// counter.  The host lists a step as the row items of domain groups A and B, then their
// column items in the same order (groups of about equal work, larger domains first in
// each), so that an item's dependencies were taken a group-phase earlier and are usually
// complete when it is taken.
//
// Dependencies, per domain only (no grid-wide barrier): a row item of step s needs every
// column item of step s - 1 of its domain done (it reads the column pass's output G and
// overwrites Rr, which that column pass read); a column item of step s needs every row item
// of step s of its domain done (it reads Rr and overwrites G).  Each domain has two
// completion counters (row items done, column items done) that only grow during a launch.
// A block about to run an item waits, in one thread, until the counter reaches the item's
// requirement (acquire loads), and after the item one thread adds 1 to its own counter
// (release).  Items are taken in increasing order and every dependency points to a smaller
// index, so the waited-for items were taken by blocks that are running: no deadlock without
// co-residency guarantees.  Every wait is bounded in time (limit_ns: 2 s in production); one
// that runs out sets the domain's status word (TTSH_E_TIMEOUT at its next synchronising call)
// and an abort flag that makes every block stop taking items.
//
// The item bodies are the single-domain row and column pass bodies with each size's
// default tile shape, so every domain's results are bit-identical to ttsh_step.  The block
// size is the largest body's; a smaller body runs on its first NT threads (its barriers are
// named barriers counting NT) while the others wait at the kernel's own barrier.
#pragma once

#include "ttsh_kernels.cuh"

namespace ttsh {

struct PItem {
  int dom;     // index into the domain table
  int phase;   // 0 = row pass, 1 = column pass
  int blk;     // block index within the pass
  int pad;
};

template <typename T>
struct PDomain {
  Args<T> A;
  int n;
  int nrow;   // row-pass blocks per step
  int ncol;   // column-pass blocks per step
  int pad;
};

// An item as the body threads read it: its list entry, its domain's grid size and argument
// block, copied into shared memory by the control lane while the previous item runs (so the
// body starts without a global-memory round trip).
template <typename T>
struct PStaged {
  Args<T> A;
  PItem it;
  int n;
};

// Control block, zeroed before every launch: [0] next item, [1] abort flag, then per domain
// [2 + 2d] row items done, [3 + 2d] column items done.
constexpr int kPersistCtlHead = 0, kPersistCtlAbort = 1, kPersistCtlDone = 2;

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// Orders this thread's generic-proxy view of global memory with the bulk copies
// (async proxy) it issues afterwards.
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Wait until *ctr >= need (acquire), the abort flag is raised, or limit_ns have passed.
__device__ __forceinline__ bool wait_count(const unsigned long long* ctr, unsigned long long need,
                                           const unsigned long long* abort_flag, unsigned long long limit_ns) {
  if (ld_acquire_u64(ctr) >= need) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    __nanosleep(64);
    if (ld_acquire_u64(ctr) >= need) return true;
    if (ld_relaxed_u64(abort_flag)) return false;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

// Sizes the persistent kernel holds (the batched sweeps' grids and smaller).
constexpr int kPersistMaxN = 512;

template <typename T, int N>
struct PersistShape {
  static constexpr int R = default_step_rows<T, N>();
  static constexpr int RPE = default_step_row_pe<T, N>();
  static constexpr int CPE = default_step_col_pe<T, N>();
  using RG = RowGeo<T, N, ROW_STEP, R, RPE>;
  using CG = ColGeo<T, N, COL_STEP, CPE>;
  static constexpr int NT = cmax(RG::NT, CG::NT);
  static constexpr int SMEM = cmax(RG::SMEM, CG::SMEM);
};

template <typename T>
struct PersistLimits {
  template <int N>
  using S = PersistShape<T, N>;
  static constexpr int NT = cmax(cmax(cmax(S<16>::NT, S<32>::NT), cmax(S<64>::NT, S<128>::NT)),
                                 cmax(S<256>::NT, S<512>::NT));
  static constexpr int SMEM = cmax(cmax(cmax(S<16>::SMEM, S<32>::SMEM), cmax(S<64>::SMEM, S<128>::SMEM)),
                                   cmax(S<256>::SMEM, S<512>::SMEM));
};

// One item's body, each size and pass a function of its own (not inlined): every body keeps
// the register allocation it has in its own kernel instead of the union of all of them.
// The argument block is copied out of the domain table first (as the per-launch batched
// kernels do), so the body's constants live in registers rather than being reloaded from
// global memory after every store.
template <typename T, int N>
__device__ __noinline__ void persist_row(const Args<T>& Ag, int blk, unsigned char* smem) {
  using S = PersistShape<T, N>;
  if (threadIdx.x < S::RG::NT) {
    const Args<T> A = Ag;
    row_body<T, N, ROW_STEP, S::R, S::RPE, 1, 0, false>(A, blk, smem, nullptr);
  }
}
template <typename T, int N>
__device__ __noinline__ void persist_col(const Args<T>& Ag, int blk, unsigned char* smem) {
  using S = PersistShape<T, N>;
  if (threadIdx.x < S::CG::NT) {
    const Args<T> A = Ag;
    col_body<T, N, COL_STEP, S::CPE>(A, blk, smem);
  }
}
template <typename T, int N>
__device__ __forceinline__ void persist_item(const Args<T>& A, int phase, int blk, unsigned char* smem) {
  if (phase == 0) persist_row<T, N>(A, blk, smem);
  else persist_col<T, N>(A, blk, smem);
}

// Requirement of item it of step st: the counter it waits on and the count it needs.
template <typename T>
__device__ __forceinline__ void item_need(const PDomain<T>* doms, const PItem& it, long long st,
                                          unsigned long long* ctl, unsigned long long** ctr,
                                          unsigned long long* need) {
  const PDomain<T>& D = doms[it.dom];
  *ctr = &ctl[kPersistCtlDone + 2 * it.dom + (it.phase == 0 ? 1 : 0)];
  *need = it.phase == 0 ? (unsigned long long)st * D.ncol : (unsigned long long)(st + 1) * D.nrow;
}

// Block = NB body threads (the largest body's thread count) + one control warp.  The control
// warp's first lane takes the next item and checks its dependency while the body threads run
// the current item, and sends the current item's completion signal while they run the next:
//   body threads:  run item g                          | barrier B | run item g' ...
//   control lane:  signal g-, take g', poll its counter | barrier B | signal g ...
// The poll during the body is relaxed and stops when the counter is high enough (then one
// acquire fence, and g' is published before barrier B: the fast path) or when the body's
// first thread reports it is done.  If g' is not ready by then, the control lane signals g
// first, then waits for g' (which may depend on g) and publishes it behind one more barrier.
// Published items alternate between two slots, so a slot is never rewritten while a thread
// may still read it.
template <typename T>
__global__ void __launch_bounds__(PersistLimits<T>::NT + 32, sizeof(T) == 4 ? 5 : 2)
persistent_step_kernel(const PDomain<T>* __restrict__ doms, const PItem* __restrict__ items, int ips,
                       long long nsteps, unsigned long long* __restrict__ ctl, unsigned long long limit_ns) {
  constexpr int NB = PersistLimits<T>::NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* smem = smem_base128(smem_raw);
  __shared__ long long s_item[2];
  __shared__ int s_fast[2];
  __shared__ PStaged<T> s_st[2];
  __shared__ volatile long long s_body_done;   // the last item whose body thread 0 finished
  const long long total = nsteps * (long long)ips;
  const bool ctrl = threadIdx.x == NB;
  unsigned long long* abort_flag = &ctl[kPersistCtlAbort];

  // the control lane's bounded wait; on a time-out the domain's status word and the abort
  // flag are raised and the block stops
  auto wait_ready = [&](const PItem& it, long long g) -> bool {
    unsigned long long* ctr;
    unsigned long long need;
    item_need(doms, it, g / ips, ctl, &ctr, &need);
    if (wait_count(ctr, need, abort_flag, limit_ns)) return true;
    atomicExch(doms[it.dom].A.err, 1);
    atomicExch(abort_flag, 1ull);
    return false;
  };
  auto take = [&]() -> long long {
    const long long g = (long long)atomicAdd(&ctl[kPersistCtlHead], 1ull);
    return (g >= total || ld_relaxed_u64(abort_flag)) ? -1 : g;
  };
  // control lane: copy item g's record, size and arguments into staging slot sl
  auto stage = [&](long long g, int sl) {
    const PItem it = items[g % ips];
    s_st[sl].it = it;
    s_st[sl].n = doms[it.dom].n;
    s_st[sl].A = doms[it.dom].A;
  };

  unsigned long long* pending = nullptr;   // control lane: the completion signal still to send
  if (ctrl) {
    long long g = take();
    if (g >= 0) stage(g, 0);
    if (g >= 0 && !wait_ready(items[g % ips], g)) g = -1;
    fence_proxy_async_global();   // the column pass reads Rr with bulk copies
    s_item[0] = g;
    s_body_done = -1;
  }
  __syncthreads();
  for (int slot = 0;; slot ^= 1) {
    const long long g = s_item[slot];
    if (g < 0) {
      if (pending) red_release_add_u64(pending, 1ull);
      return;
    }
    const PItem it = s_st[slot].it;
    long long gn = -1;
    bool ready = false;
    if (threadIdx.x < NB) {
      const Args<T>& A = s_st[slot].A;
      switch (s_st[slot].n) {
        case 16: persist_item<T, 16>(A, it.phase, it.blk, smem); break;
        case 32: persist_item<T, 32>(A, it.phase, it.blk, smem); break;
        case 64: persist_item<T, 64>(A, it.phase, it.blk, smem); break;
        case 128: persist_item<T, 128>(A, it.phase, it.blk, smem); break;
        case 256: persist_item<T, 256>(A, it.phase, it.blk, smem); break;
        case 512: persist_item<T, 512>(A, it.phase, it.blk, smem); break;
        default: break;
      }
      if (threadIdx.x == 0) s_body_done = g;   // a hint for the control lane's poll
    } else if (ctrl) {
      if (pending) {   // the previous item's signal, sent while this one runs
        red_release_add_u64(pending, 1ull);
        pending = nullptr;
      }
      gn = take();
      if (gn >= 0) {
        stage(gn, slot ^ 1);   // slot ^ 1 was read by the previous item, which is done
        unsigned long long* ctr;
        unsigned long long need;
        item_need(doms, items[gn % ips], gn / ips, ctl, &ctr, &need);
        while (!(ready = ld_relaxed_u64(ctr) >= need) && s_body_done != g) __nanosleep(256);
        if (ready) {
          asm volatile("fence.acq_rel.gpu;" ::: "memory");
          fence_proxy_async_global();   // the column pass reads Rr with bulk copies
        }
      }
      // fast path: publish the next item before barrier B (also when there is none)
      const bool fast = gn < 0 || ready;
      s_fast[slot] = fast ? 1 : 0;
      if (fast) s_item[slot ^ 1] = gn;
      pending = &ctl[kPersistCtlDone + 2 * it.dom + it.phase];
    }
    __syncthreads();   // B: the item's stores are issued; the next item is known
    if (!s_fast[slot]) {   // uniform: the next item waits for a dependency (possibly this item)
      if (ctrl) {
        red_release_add_u64(pending, 1ull);
        pending = nullptr;
        if (!wait_ready(items[gn % ips], gn)) gn = -1;
        fence_proxy_async_global();
        s_item[slot ^ 1] = gn;
      }
      __syncthreads();
    }
  }
}

}  // namespace ttsh
