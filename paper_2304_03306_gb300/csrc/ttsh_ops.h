// ttsh_ops.h - precision-erased launch interface between the host runtime (ttsh_api.cu)
// and the per-precision kernel translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ttsh {

// Device pointers and constants of one domain, independent of the arithmetic type.
struct DomainDev {
  void* what;      // omega^ half-spectrum, H x NK complex
  void* vmean;     // v^(0), 2 reals
  void* K;         // processed mask, N x N reals
  void* G;         // [3][H][N] complex
  void* Rr;        // [3][H][N] complex
  void* tw;        // N complex twiddles W_N^m
  double* real;    // [3][N][N] double staging
  double* part;    // row-block diagnostic partials
  double* colhist; // H x (N/4 + 1) spectrum partials
  int* bad;        // non-finite counter
  double* out;     // reduced diagnostics (8 doubles: 5 sums, 2 divergence maxima, 1 spare) + spectrum bins
  unsigned char* knaive;   // binary mask K_naive as given (1 = masked), N x N bytes
  double* rec;     // time-series partials of a recorded step (null: plain step)
  void* recctl;    // time-series write position (RecCtl), used with rec
  double a, b, lam, gv, gw, dx, dt;
  double cx, cy;   // centre for the order parameter
  int n;
  int pdl;         // launch the step kernels with programmatic dependent launch
  int use_tma;     // let the row step kernel load its G tile with the TMA (where tma_ok)
  int* err;        // device status word (bounded waits that ran out)
  // G as a 2D tensor for the row pass's TMA loads, one map per row-block height R = 1, 2, 4
  // (tma_ok[i] = 0 where the shape does not allow it or the map could not be made)
  CUtensorMap tmapG[3];
  int tma_ok[3];
};

enum { K_ROW_STEP = 0, K_ROW_FWD_VEL = 1, K_ROW_FWD_MASK = 2, K_ROW_INV_FIELDS = 3,
       K_ROW_INV_MASK = 4, K_ROW_INV_DIAG = 5 };
enum { K_COL_STEP = 0, K_COL_PROLOGUE = 1, K_COL_PROJECT = 2, K_COL_MASK = 3, K_COL_ADDW = 4, K_COL_DIV = 5 };

using RowFn = cudaError_t (*)(int kind, const DomainDev&, cudaStream_t);
using ColFn = cudaError_t (*)(int mode, const DomainDev&, cudaStream_t);
using SpecFn = cudaError_t (*)(const DomainDev&, int nbins, cudaStream_t);
using BlocksFn = int (*)(int kind);

using StepFn = cudaError_t (*)(const DomainDev&, cudaStream_t);
// Batched launch: `args` is a device array of ndom per-domain kernel argument blocks.
using BatchFn = cudaError_t (*)(const void* args, int ndom, cudaStream_t);
using PrepareFn = cudaError_t (*)();

// One tile shape of a step kernel: rows per block (row pass only) and points per thread of
// the register butterflies.  `batched` / `prepare` are set for grids up to kMaxBatchN.
struct StepVariant {
  StepFn fn;
  BatchFn batched;
  PrepareFn prepare;   // sets the batched kernel's attributes (call before graph capture)
  int rows;
  int pe;
  int cl;    // blocks per cluster (row pass)
  int cmp;   // 1: compact row pass (in-place forward transforms)
  int tma;   // 1: the row pass can stage its G tile by TMA (launch mode bit 1)
};

constexpr int kMaxBatchN = 1024;

constexpr int kMaxVariants = 12;

struct SizeOps {
  RowFn row;
  ColFn col;
  SpecFn spec;
  BlocksFn row_blocks;   // grid size of a row kernel kind (number of diagnostic partials)
  int n_row_variants, n_col_variants;           // entry 0 is the default tile shape
  StepVariant row_step[kMaxVariants];
  StepVariant col_step[kMaxVariants];
  int args_bytes;                                    // size of one kernel argument block
  void (*pack_args)(const DomainDev&, void* dst);    // host copy of a domain's argument block
};

// Persistent batched stepper of one precision (ttsh_persist_*.cu): one launch advances a
// batch of domains with n <= max_n (each with its size's default tile shape) by nsteps.
struct PersistOps {
  // doms: device table of ndom packed domains (domain_bytes each); items: device list of
  // ips work items (item_bytes each); ctl: 2 + 2 ndom zeroed 64-bit counters
  cudaError_t (*launch)(const void* doms, const void* items, int ips, long long nsteps,
                        unsigned long long* ctl, int grid, unsigned long long limit_ns, cudaStream_t s);
  cudaError_t (*prepare)(int* grid);   // kernel attributes; resident blocks on this device
  void (*pack)(const DomainDev& d, int nrow, int ncol, void* dst);
  int (*row_blocks)(int n);            // row-pass blocks per step of size n (0: not held)
  int domain_bytes, item_bytes;
  int max_n;
  int threads;                         // block size
};
bool persist_f32(PersistOps* o);
bool persist_f64(PersistOps* o);

// Per translation unit registries; return false if the TU does not hold size n.
bool ops_f32_small(int n, SizeOps* o);
bool ops_f32_large(int n, SizeOps* o);
bool ops_f64_small(int n, SizeOps* o);
bool ops_f64_large(int n, SizeOps* o);

// Record the calling thread's message for ttsh_last_error() (used by entry points defined
// outside ttsh_api.cu).
void set_last_error(const char* msg);
void set_last_error(const char* what, cudaError_t e);

}  // namespace ttsh

struct ttsh_domain;
namespace ttsh {
// Accessors used by the corrector (ttsh_fno.cu) to work on a domain's device state.
const DomainDev* domain_dev(const ttsh_domain* d);
cudaStream_t domain_stream(const ttsh_domain* d);
int domain_precision(const ttsh_domain* d);
int domain_n(const ttsh_domain* d);
double domain_dx(const ttsh_domain* d);
// Real-space omega, v_x, v_y of the state into the domain's double staging planes 0..2.
int domain_fields_to_staging(ttsh_domain* d);
// Add the real field in staging plane 0 to omega (projected onto the 1/2-rule disc,
// Hermitian, zero mean) and refresh the inter-pass buffers.
int domain_add_vorticity_from_staging(ttsh_domain* d);
// Adjust the step counter (for steps replayed from a graph the domain did not record).
void domain_add_steps(ttsh_domain* d, int64_t n);
double domain_dt(const ttsh_domain* d);
// Rebuild the inter-pass buffers from the spectral state (after writing it on the device).
int domain_refresh(ttsh_domain* d);
int domain_refresh_on(ttsh_domain* d, cudaStream_t s);   // on another stream (graph capture)
// Copy of a domain (parameters, mask, plan, stream, state) in a new library-owned workspace.
int domain_clone(const ttsh_domain* src, ttsh_domain** out);

cudaError_t launch_diag_reduce(const double* part, int nblocks, double* out, cudaStream_t s);
cudaError_t launch_spectrum_reduce(const double* colhist, int ncols, int nbins, double scale,
                                   double* out, cudaStream_t s);

}  // namespace ttsh
