/*
 * ttsh.h - C ABI of the GB300 (sm_103a) solver for the confined Toner-Tu-Swift-Hohenberg
 * (TTSH) polar-active-fluid model of arXiv:2304.03306.
 *
 * The model is the vorticity form of the TTSH equation with damping mask K(x), Eq. (mod1)-
 * (mod2) (Sec. II.A), with the constants of Table I.  A domain is one N x N periodic box
 * (L = N dx) whose boundary is given only as a binary mask K_naive (Sec. II.C); the library
 * turns it into the band-limited, non-negative K of Algorithm 2 (Appendix E) and time-steps
 * the state with the pseudospectral integrating-factor Euler scheme of Algorithm 1
 * (Appendix D).  All arithmetic of a step runs in this library's CUDA kernels.
 *
 * Conventions shared by every entry point:
 *  - Real fields are N*N arrays indexed [y][x] (row-major), grid point (i, j) at
 *    x = (j - N/2) dx, y = (i - N/2) dx.
 *  - The DFT is the unitary one of Appendix D: f^(k) = N^-1 sum_x f(x) e^{-i k.x}, inverse
 *    with e^{+i k.x} and N^-1; k = dk * m, dk = 2 pi / (N dx), m integer.
 *  - The spectral state omega^ is stored as the Hermitian half-spectrum restricted to the
 *    1/2-rule disc: columns mx = 0..N/4 ("H = N/4 + 1" columns), each holding
 *    "NK = N/2 + 1" values for my = 0..N/4 then my = -N/4..-1 (entry j <-> my = j for
 *    j <= N/4, my = j - NK otherwise).  Modes with mx^2 + my^2 > (N/4)^2 are zero.  The
 *    spatial mean velocity v^(0) (two reals, unitary DFT at k = 0, i.e. N * mean) is kept
 *    separately, as Algorithm 1 does at k = 0.
 *  - Host pointers are owned by the caller and are only read/written during the call.
 *  - Every call returns a ttsh_status; no C++ exception crosses the ABI.  A thread-local
 *    message for the last failure is returned by ttsh_last_error().
 *  - Kernels run on the domain's stream.  ttsh_step is asynchronous; calls that return
 *    host data synchronise the stream first.  A device-side failure surfaces as
 *    TTSH_E_CUDA at the next synchronising call.  Every wait inside a kernel (TMA and
 *    bulk-copy completion, tensor-core completion) is bounded; one that runs out sets a
 *    status word that ttsh_synchronize / ttsh_diagnostics report as TTSH_E_TIMEOUT.
 */
#ifndef TTSH_H
#define TTSH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TTSH_OK = 0,
  TTSH_E_INVALID = 1,      /* bad argument (size, pointer, parameter value)              */
  TTSH_E_OOM = 2,          /* device allocation failed                                    */
  TTSH_E_CUDA = 3,         /* a CUDA runtime call or kernel failed                        */
  TTSH_E_TIMEOUT = 4,      /* a bounded wait inside a kernel ran out                      */
  TTSH_E_NONFINITE = 5,    /* the state holds NaN or Inf (reported by ttsh_diagnostics)   */
  TTSH_E_UNSUPPORTED = 6   /* a valid request this build does not implement              */
} ttsh_status;

/* Model and discretisation constants.  Defaults (ttsh_default_params) are Table I:
 * a = 0.5, b = 1.6, lambda = 9, gamma_v = 40, gamma_w = 4, dt = 0.01, N = 8192, dx = 0.005.
 * n must be a power of two in [16, 8192]; precision is 32 (float) or 64 (double) and
 * selects the arithmetic of every kernel of the domain.  Double precision has kernels up to
 * n = 4096 (one row of three double fields at 8192 exceeds a block's shared memory);
 * ttsh_create_domain returns TTSH_E_UNSUPPORTED for n = 8192 with precision 64. */
typedef struct {
  double a, b, lambda, gamma_v, gamma_w;
  double dx, dt;
  int32_t n;
  int32_t precision;
} ttsh_params;

/* Observables of the current state, accumulated in double precision whatever the
 * domain precision (sums in a fixed order, so repeated calls give identical bits):
 *   energy    = (2 N^2)^-1 sum_x |v|^2
 *   enstrophy = (2 N^2)^-1 sum_x omega^2
 *   psi       = vortex order parameter of Sec. III.C: (sum|e_theta.v| / sum|v| - 2/pi)
 *               / (1 - 2/pi) over every grid point, about the given centre (e_theta := 0
 *               at the centre itself)
 *   max_div   = max |k.v^(m)| / max |k| |v^(m)| over the modes of the 1/2-rule disc, where
 *               v^ = DFT[v] of the real-space velocity the row pass works with (the
 *               incompressibility div v = 0 that the stream-function construction of
 *               Appendix D guarantees; round-off level: ~1e-16 double, ~1e-7 float)
 *   mean_vx, mean_vy = spatial mean of v (= v^(0) / N)
 *   nonfinite = number of non-finite values met in the state's real-space fields. */
typedef struct {
  double energy, enstrophy, psi, max_div, mean_vx, mean_vy;
  int64_t step;
  int32_t nonfinite;
  int32_t reserved;
} ttsh_diag;

typedef struct ttsh_domain ttsh_domain;
typedef struct ttsh_batch ttsh_batch;
typedef struct ttsh_fno ttsh_fno;

/* Fill *p with the Table I constants (Appendix B).  Never fails. */
void ttsh_default_params(ttsh_params* p);

/* Bytes of device memory one domain with these parameters uses (state, mask, the two
 * inter-pass buffers, staging and reduction scratch, twiddle table), or 0 if the
 * parameters are invalid.  Passing a caller-owned block of at least this size (256-byte
 * aligned) to ttsh_create_domain makes the library allocate nothing. */
size_t ttsh_workspace_bytes(const ttsh_params* p);

/* Create a domain from a binary mask (Sec. II.C; Algorithm 2 of Appendix E runs on the
 * GPU: DFT, zero |m|^2 > (N/8)^2, inverse DFT, square).
 *   mask       host, N*N bytes [y][x]; nonzero = masked (K_naive = 1), 0 = inside.
 *   p          parameters; validated (n power of two in [16, 8192], dx > 0, dt > 0,
 *              precision 32 or 64) -> TTSH_E_INVALID otherwise; n = 8192 with precision
 *              64 -> TTSH_E_UNSUPPORTED.
 *   workspace  device pointer of ttsh_workspace_bytes(p) bytes owned by the caller (it
 *              must outlive the domain), or NULL to let the library cudaMalloc it.
 *   stream     cudaStream_t the domain's kernels are issued on (NULL = legacy default).
 *   out        receives the handle.
 * The state starts at zero (omega^ = 0, v^(0) = 0). */
ttsh_status ttsh_create_domain(const uint8_t* mask, const ttsh_params* p, void* workspace,
                               void* stream, ttsh_domain** out);

/* Release the domain (and its workspace if the library allocated it).  NULL is a no-op. */
void ttsh_destroy_domain(ttsh_domain* d);

/* Change the stream later kernels are issued on; work already queued on the previous
 * stream is ordered before them by a device-side wait (the host does not block). */
ttsh_status ttsh_set_stream(ttsh_domain* d, void* stream);

/* Set the state from a real velocity field (host, N*N doubles each).  The field is
 * projected as the initial condition of the method: omega^ = i k x v^, then Algorithm 1's
 * post-processing (omega^(0) = 0, v^(0) = DFT[v](0), zero |m|^2 > (N/4)^2, Hermitian
 * average, v from the stream function), so the stored state is divergence-free and
 * band-limited.  Resets the step counter. */
ttsh_status ttsh_set_velocity(ttsh_domain* d, const double* vx, const double* vy);

/* Same, from a real velocity field already on the device (N*N doubles each, any
 * 8-byte-aligned device pointers, read during the call only). */
ttsh_status ttsh_set_velocity_device(ttsh_domain* d, const double* vx, const double* vy);

/* Set the state to the paper's "random initial state" (Sec. III.A and Sec. IV.A), generated
 * on the device: at every point inside the domain (mask byte 0 in the mask given to
 * ttsh_create_domain) v_x and v_y are independent draws, uniform on [-amplitude, amplitude),
 * and 0 at masked points; then projected as ttsh_set_velocity does.  The draws come from
 * the SplitMix64 generator (Steele, Lea & Flood 2014) in counter form: at flattened point
 * p = y N + x, v_x uses output 2p and v_y output 2p + 1 of the stream seeded with `seed`,
 * an output z giving u = (z >> 11) 2^-53 and the value amplitude (2u - 1) in double
 * precision.  The same seed therefore gives the same field, bit for bit, as any other
 * implementation of that definition, on any grid size.  amplitude must be finite
 * (TTSH_E_INVALID otherwise).  Resets the step counter; synchronises. */
ttsh_status ttsh_init_noise(ttsh_domain* d, uint64_t seed, double amplitude);

/* Advance the state by nsteps steps of the pseudospectral integrating-factor Euler scheme
 * of Appendix D (Algorithm 1) for Eq. (mod2): the real-space non-linear and mask terms (the
 * advection v.grad(omega) is evaluated in its conservative form div(v omega), which equals
 * it on every kept mode up to rounding because v and omega are band-limited to the
 * 1/2-rule disc and div v = 0), the DFT of those terms and their curl, the integrating-
 * factor Euler update omega^ <- exp((a - (1 - k^2)^2) dt)(omega^ + dt rhs^), the k = 0
 * mean-flow update of Eq. (avg), the 1/2-rule dealiasing, the Hermitian average and the
 * stream-function velocity.  Asynchronous on the domain's stream; long runs are replayed as
 * CUDA graphs.  nsteps < 0 -> TTSH_E_INVALID; 0 is a no-op. */
ttsh_status ttsh_step(ttsh_domain* d, int64_t nsteps);

/* Copy the real-space fields of the current state to the host (N*N doubles each, [y][x]):
 * v_x, v_y (including the mean flow) and omega = iDFT[omega^].  Any pointer may be NULL. */
ttsh_status ttsh_get_fields(ttsh_domain* d, double* vx, double* vy, double* omega);

/* Copy the processed mask K of Algorithm 2 (N*N doubles, [y][x]) to the host. */
ttsh_status ttsh_get_mask(ttsh_domain* d, double* K);

/* Checkpoint / resume of the exact state: omega^ as interleaved (re, im) doubles in the
 * half-spectrum layout described above (H * NK complex values, column mx-major), and
 * v^(0) as 2 doubles.  set_spectral_state converts to the domain precision (exact for a
 * state read back from a domain of the same precision, so a resumed run is bit-identical)
 * and does not alter the values (no re-projection). */
ttsh_status ttsh_get_spectral_state(ttsh_domain* d, double* w_hat, double* v0);
ttsh_status ttsh_set_spectral_state(ttsh_domain* d, const double* w_hat, const double* v0);

/* Diagnostics of the current state (see ttsh_diag).  centre: (x, y) of the centre used by
 * psi, NULL = (0, 0).  spectrum: if non-NULL, receives nbins doubles of the shell energy
 * spectrum E(s) = (2 N^2)^-1 sum over modes with round(|m|) = s of |v^(m)|^2; shells beyond
 * N/4 are zero.  nbins must be in [0, 65536].  Synchronises.  Returns TTSH_E_NONFINITE
 * (with *out filled) when the state holds NaN/Inf. */
ttsh_status ttsh_diagnostics(ttsh_domain* d, ttsh_diag* out, double* spectrum, int32_t nbins,
                             const double* centre);

/* Advance nsteps steps (as ttsh_step) while recording a time series of the observables of
 * Sec. III.C without synchronising: the state at step counts s0, s0 + every, s0 + 2 every,
 * ... (s0 = step count at the call; one sample per started block of `every` steps, so
 * ceil(nsteps / every) samples) is sampled inside that step's row pass, which already holds
 * omega, v_x and v_y in real space.  Sample j is written to series[5 j .. 5 j + 4] =
 * {step count, energy, enstrophy, psi, number of non-finite points}, with the definitions of
 * ttsh_diag; per-thread, per-warp and per-block partial sums are taken in the domain
 * precision and the blocks' sums combined as double-float pairs (float domains) or in double,
 * all in a fixed order (repeatable bits).  To record the state after the last step, call
 * ttsh_diagnostics afterwards.
 *   every     >= 1 steps between samples.
 *   series    device (or managed) memory of at least 5 * capacity doubles, owned by the
 *             caller; it must stay valid until the stream has passed the call.
 *   capacity  samples series can hold; smaller than ceil(nsteps / every) -> TTSH_E_INVALID
 *             (nothing is stepped).
 *   centre    (x, y) for psi, NULL = (0, 0).
 * Asynchronous on the domain's stream; replayed as CUDA graphs of every * floor(64 / every)
 * steps when every <= 64.  The paper has no counterpart of this entry point: it is the
 * device-side form of the energy / order-parameter time series its runs record. */
ttsh_status ttsh_step_record(ttsh_domain* d, int64_t nsteps, int32_t every, double* series,
                             int64_t capacity, const double* centre);

/* Kernel timing for roofline reports: records `iters` back-to-back launches of the row pass
 * (then of the column pass) of the current plan as CUDA graphs, replays them between CUDA
 * events on the domain's stream and writes the mean duration of one launch in milliseconds
 * to ms[0] (row pass) and ms[1] (column pass).  The launches are ordinary ones whatever the
 * domain's launch mode, so each duration is a whole launch.  The spectral state is saved
 * before and restored after, so the domain continues exactly where it was.  Synchronises.
 * iters must be in [1, 1000000]. */
ttsh_status ttsh_time_kernels(ttsh_domain* d, int32_t iters, double* ms);

/* Step-kernel tile shapes ("plan").  Each grid size has a list of row-pass variants (rows
 * per block, points per thread of the register butterflies) and column-pass variants
 * (points per thread); entry 0 is the default.  Variants compute the same step with a
 * different factorisation of the transforms, so results agree to rounding, not bit for bit.
 * ttsh_autotune times every variant (as ttsh_time_kernels does, `iters` launches each, state
 * restored) and selects the fastest row and column variant.  plan (10 int32, may be NULL):
 * {row variant, column variant, rows per block, row points per thread, column points per
 * thread, number of row variants, number of column variants, launch mode, row blocks per
 * cluster, compact row pass}.  On grids of 2048^2 and more, float row variants with two
 * blocks per cluster stage the column-major inter-pass tiles for both blocks' rows at once
 * and swap halves through distributed shared memory.  On 1024^2 to 4096^2 grids, compact
 * float row variants transform in place (no separate forward buffers), so that two blocks
 * fit per SM and one block's staging and stores overlap the other's transforms.  ttsh_set_plan
 * selects variants by index (TTSH_E_INVALID if out of range).  ttsh_autotune times each row
 * variant with its G tile staged both ways where it can be (see ttsh_set_launch_mode), keeps the fastest
 * (variant, staging) pair, and then times whole steps (graphs of up to 64 steps, state
 * restored) with and without programmatic dependent launch and keeps the faster. */
ttsh_status ttsh_autotune(ttsh_domain* d, int32_t iters, int32_t* plan);
ttsh_status ttsh_get_plan(ttsh_domain* d, int32_t* plan);
ttsh_status ttsh_set_plan(ttsh_domain* d, int32_t row_variant, int32_t col_variant);

/* Launch mode of the step kernels, a bit set:
 *   bit 0  programmatic dependent launches: a pass may start (copy its twiddle tables and
 *          mask rows) while the previous pass is still running and waits on the device
 *          (griddepcontrol.wait) before it reads anything that pass wrote;
 *   bit 1  the row pass loads its G tile with the tensor-memory accelerator (one 2D tile load
 *          per field, completion on an mbarrier with a bounded wait) instead of cp.async,
 *          where the tile allows it (N <= 512, a row segment of R complex values a multiple
 *          of 16 bytes, and a dense tile: variants whose staged tile has a spare slot per
 *          column against shared-memory bank conflicts do not qualify); elsewhere cp.async
 *          is used whatever the bit.
 * Results are bit-identical in every mode; values outside [0, 3] -> TTSH_E_INVALID.  The
 * paper has no counterpart: these are scheduling options. */
ttsh_status ttsh_set_launch_mode(ttsh_domain* d, int32_t mode);

/* Advance a caller-owned state by nsteps steps of Algorithm 1 without allocating any device
 * memory (the paper has no counterpart: this is a library convenience).  It is meant for
 * callers that cannot let a library call cudaMalloc - their device memory belongs to their
 * own pool or fixed budget, or they cannot afford the device-wide synchronisation an
 * allocation or free implies.  Inputs and outputs are the caller's device buffers, in the
 * precision p->precision selects (float or double):
 *   K      N*N mask values [y][x] (e.g. copied from ttsh_get_mask), read only;
 *   w_hat  omega^ in the half-spectrum layout above, H*NK complex (re, im interleaved),
 *          advanced in place;
 *   v0     v^(0), 2 values, advanced in place.
 * All three must be 16-byte aligned (as cudaMalloc's are); otherwise -> TTSH_E_INVALID,
 * before any device work.
 * Scratch (inter-pass buffers, twiddle tables) lives in one fixed device array inside the
 * library, sized for n <= 512 (about 6.4 MB, held by every GPU that loads the library until
 * the process exits); n > 512 -> TTSH_E_INVALID, as are the parameter checks of
 * ttsh_create_domain.  The first call on each device resolves that array's address, writes
 * its twiddle tables and waits for the whole device (cudaDeviceSynchronize) so that the
 * tables are in place before any kernel on any stream reads them; make that first call
 * before any stream capture.  All calls share the array, so calls that overlap on the GPU
 * race: serialise them.  Kernels are issued on `stream` (NULL = legacy default) and the call
 * returns without waiting for them.  A bounded wait inside the kernels that ran out (a lost
 * bulk-copy completion) is not reported by this entry point; the domain path reports it as
 * TTSH_E_TIMEOUT. */
ttsh_status ttsh_step_noalloc(const ttsh_params* p, const void* K, void* w_hat, void* v0,
                              int64_t nsteps, void* stream);

/* Lyapunov exponents of a domain's trajectory (Sec. III.C: growth rates of independent
 * perturbations delta omega_i evolved along with omega, obtained from QR decompositions as in
 * Shimada & Nagashima 1979 and Benettin et al. 1980).  The paper does not say how the
 * perturbations are evolved; here each is a copy of the domain started at base + eps q_i and
 * stepped with it (batched with it for n <= 1024), so a perturbation evolves as the finite
 * difference (copy - base) / eps of the scheme of Algorithm 1.  After every `interval` steps
 * the k differences are re-orthonormalised by classical Gram-Schmidt applied twice, in
 * double precision, log R_ii is accumulated and the copies are reset to base + eps q_i.
 * State vectors (D = 2 H NK + 2 doubles, H = N/4 + 1, NK = N/2 + 1) are omega^ in the stored
 * half-spectrum layout (interleaved re/im, as ttsh_get_spectral_state) followed by v^(0); the
 * inner product weights the mx > 0 columns by 2 (they stand for +-mx), which makes it the
 * real-space sum_x omega omega' plus v^(0).v'^(0).
 *   create   base: the domain whose trajectory is analysed (it is stepped by ttsh_lyap_step);
 *            k in [1, 16] perturbations; eps > 0 their size in that norm; q0: host, k x D
 *            doubles, the initial directions (orthonormalised on the device; they should be
 *            Hermitian in the mx = 0 column and zero outside the 1/2-rule disc, as a state is).
 *            The copies use k extra domain workspaces.  Synchronises.
 *   step     advance base and copies by nsteps (a multiple of interval; interval fixed for
 *            the run) with a renormalisation after every interval.  Asynchronous.
 *   result   exponents[k] = accumulated log R_ii / elapsed time, largest first in the limit;
 *            last_rates[k] (may be NULL) = log R_ii / (interval dt) of the last interval.
 *            TTSH_E_INVALID before the first interval.  Synchronises.
 *   directions  the current orthonormal directions q_i (host, k x D doubles).  Synchronises.
 * Not in the paper's interface: these entry points are this library's form of its Lyapunov
 * analysis. */
typedef struct ttsh_lyap ttsh_lyap;
ttsh_status ttsh_lyap_create(ttsh_domain* base, int32_t k, double eps, const double* q0, ttsh_lyap** out);
ttsh_status ttsh_lyap_step(ttsh_lyap* L, int64_t nsteps, int32_t interval);
ttsh_status ttsh_lyap_result(ttsh_lyap* L, double* exponents, double* last_rates);
ttsh_status ttsh_lyap_directions(ttsh_lyap* L, double* q);
void ttsh_lyap_destroy(ttsh_lyap* L);

/* Batched stepping of many independent domains, as the paper's radius and dumbbell sweeps
 * (Sec. III.C, Sec. IV) need: dozens of small domains of uneven sizes advanced together.
 * ttsh_batch_create groups the domains by (precision, n, plan); every group advances in one
 * launch per pass (row, column) for all its domains, and the groups run as parallel branches
 * of one CUDA graph replayed 32 steps at a time.  Each domain's result is bit-identical to
 * ttsh_step on that domain alone.
 *   domains  ndom distinct handles (ndom >= 1), each with n <= 1024 (TTSH_E_UNSUPPORTED
 *            otherwise); they must outlive the batch and are not copied.  The plan each
 *            domain has at creation is used; later ttsh_set_plan calls do not affect it.
 *   stream   stream the batch is issued on (NULL = legacy default).
 * ttsh_batch_step advances every domain by nsteps and adds nsteps to their step counters.
 * It is asynchronous: work already queued on each domain's own stream is ordered before it by
 * a device-side wait (the host does not block); whole multiples of 32 steps replay one graph,
 * and a remainder replays a graph cached for the next call with the same remainder. */
ttsh_status ttsh_batch_create(ttsh_domain* const* domains, int32_t ndom, void* stream, ttsh_batch** out);
ttsh_status ttsh_batch_step(ttsh_batch* b, int64_t nsteps);
ttsh_status ttsh_batch_synchronize(ttsh_batch* b);
int32_t ttsh_batch_groups(const ttsh_batch* b);   /* number of launch groups, -1 if NULL */

/* Persistent stepping of a batch (the default where the batch allows it): one kernel launch
 * per ttsh_batch_step call advances every domain by all nsteps steps.  The launch keeps as
 * many blocks resident as the GPU holds; they take work items - one row-pass or column-pass
 * block of one domain's step - in order from a counter, and each item waits (bounded, 2 s,
 * TTSH_E_TIMEOUT on the domain otherwise) only for the previous pass of its own domain, so
 * domains of different sizes proceed independently without a grid-wide barrier.  Needs
 * every domain in one precision, n <= 512 and the default tile shapes (plan variants 0);
 * each domain's result is bit-identical to ttsh_step.  on = 1 selects it (TTSH_E_UNSUPPORTED
 * if the batch does not allow it), 0 the grouped launches described above.
 * ttsh_batch_persistent returns 1, 0, or -1 for NULL. */
ttsh_status ttsh_batch_set_persistent(ttsh_batch* b, int32_t on);
int32_t ttsh_batch_persistent(const ttsh_batch* b);

/* Test hook of the persistent stepper's failure path (no counterpart in the paper): launches,
 * on the batch's stream, the persistent kernel with one block and a one-item work list - the
 * first column item of the first domain's first step, whose row items are not in the list - with
 * the dependency wait limited to `seconds` (0 < seconds <= 1, else TTSH_E_INVALID;
 * TTSH_E_UNSUPPORTED for a batch that cannot step persistently).  The wait runs out, sets the
 * first domain's status word and the launch's abort flag, and the block returns without
 * running the item, so the first domain's next ttsh_synchronize returns TTSH_E_TIMEOUT once;
 * no state is changed and the context and the batch stay usable.  (Production waits are
 * limited to 2 s.) */
ttsh_status ttsh_batch_test_stalled_wait(ttsh_batch* b, double seconds);
void ttsh_batch_destroy(ttsh_batch* b);           /* NULL is a no-op; domains are untouched */

/* Temporal power spectral density of the vorticity, Eq. (PSD) of Sec. III.B:
 *   S(W) = N^-2 sum_x |sum_t omega(x, t) exp(-i W t)|^2,
 * summed over the snapshots passed to ttsh_psd_accumulate.  ttsh_psd_begin sets the nfreq
 * angular frequencies W (host array, nfreq in [1, 4096]) and clears the accumulators (it
 * allocates 2 * nfreq * H * NK complex doubles plus small buffers, freed with the domain);
 * ttsh_psd_accumulate(t) adds the current state at time t (asynchronous); ttsh_psd_result
 * writes the nfreq values of S to the host (synchronises).  Computed on the spectral state
 * through Parseval in double precision, so it equals the real-space definition to rounding. */
ttsh_status ttsh_psd_begin(ttsh_domain* d, const double* omegas, int32_t nfreq);
ttsh_status ttsh_psd_accumulate(ttsh_domain* d, double t);
ttsh_status ttsh_psd_result(ttsh_domain* d, double* S);

/* Dumbbell order parameter of Sec. IV.B:
 *   Psi_2 = |omega(x*_L) + omega(x*_R)| / (|omega(x*_L)| + |omega(x*_R)|),
 * x*_{L,R} = argmax |omega| over the grid points within `radius` (= D/2, closed disc) of the
 * cavity centres (centres = {xL, yL, xR, yR}); ties go to the first point in row-major
 * order.  out[0] = Psi_2, out[1] = omega(x*_L), out[2] = omega(x*_R).  TTSH_E_INVALID if a
 * disc holds no grid point.  Double precision; synchronises. */
ttsh_status ttsh_dumbbell_order(ttsh_domain* d, const double* centres, double radius, double* out);

/* Spectral restriction of a fine domain's state onto a coarse domain covering the same box
 * (n_fine * dx_fine == n_coarse * dx_coarse, n_coarse <= n_fine, same precision): the coarse
 * unitary coefficients are the fine ones times n_coarse/n_fine on the coarse 1/2-rule disc,
 * so the coarse real-space fields are the band-limited fine fields sampled on the coarse
 * grid.  Used to build the learned corrector's training targets.  Resets the coarse step
 * counter.  Waits for the fine domain's stream, runs on the coarse domain's stream and
 * synchronises it before returning. */
ttsh_status ttsh_restrict(const ttsh_domain* fine, ttsh_domain* coarse);

/* ---------------------------------------------------------------------------------------
 * Learned corrector (not in the paper): a Fourier neural operator (Li et al., ICLR 2021)
 * that corrects the vorticity after a coarse solver step taken with a larger time step.
 *   x (B*n*n x 4): per point (omega, v_x, v_y, K) times in_scale, indexed [b][y][x][c]
 *   lift 4 -> C, then `layers` blocks z = h W + b + SpectralConv(h), h' = GELU(z) (none after
 *   the last block), projection C -> 1: the predicted omega correction times out_scale.
 *   SpectralConv keeps kx < modes and ky in {0..modes-1} U {n-modes..n-1} of rfft2(h) and
 *   mixes channels per kept mode with a complex C x C matrix, then irfft2.
 * Weights: FP32 master copies (flat vector, order: Wp[4][C], bp[C], per block Wr[2m][m][C][C],
 * Wi[2m][m][C][C], W[C][C], b[C], then Wq[C], bq) used as BF16 by the kernels, FP32
 * accumulation; channel mixing on the tensor cores.  All device pointers below are the
 * caller's (FP32).  Width must be 32 and in_channels 4 (TTSH_E_UNSUPPORTED otherwise). */
typedef struct {
  int32_t n, width, modes, layers, in_channels, max_batch;
} ttsh_fno_config;

/* Seeded initialisation (SplitMix64): pointwise weights U(-1/sqrt(fan_in), 1/sqrt(fan_in)),
 * spectral weights U(0, 1/C^2), biases 0.  Allocates its parameters and activations for up to
 * max_batch samples.  Runs on `stream`. */
ttsh_status ttsh_fno_create(const ttsh_fno_config* cfg, uint64_t seed, void* stream, ttsh_fno** out);
void ttsh_fno_destroy(ttsh_fno* f);
int64_t ttsh_fno_num_params(const ttsh_fno* f);
ttsh_status ttsh_fno_get_params(ttsh_fno* f, float* host);      /* num_params floats */
ttsh_status ttsh_fno_set_params(ttsh_fno* f, const float* host);
ttsh_status ttsh_fno_set_scales(ttsh_fno* f, const float* in_scale /* 4 */, float out_scale);
/* y (B*n*n) = network(x); asynchronous. */
ttsh_status ttsh_fno_forward(ttsh_fno* f, const float* x, float* y, int32_t batch);
/* Mean squared error of network(x) against target (B*n*n) and its gradient with respect to
 * every parameter (kept on the device for ttsh_fno_adam_step; copied to grad_host when
 * non-NULL).  Synchronises. */
ttsh_status ttsh_fno_loss_grad(ttsh_fno* f, const float* x, const float* target, int32_t batch, double* loss,
                               float* grad_host);
/* One Adam step (Kingma & Ba 2015, bias-corrected) with the last gradient. */
ttsh_status ttsh_fno_adam_step(ttsh_fno* f, float lr, float beta1, float beta2, float eps);
/* Network input of sample `sample` from a domain's current state (domain n == network n). */
ttsh_status ttsh_fno_features(ttsh_fno* f, ttsh_domain* d, float* x, int32_t sample);
/* Training target of sample `sample`: (omega(truth) - omega(base)) * out_scale. */
ttsh_status ttsh_fno_residual(ttsh_fno* f, ttsh_domain* truth, ttsh_domain* base, float* target, int32_t sample);
/* Apply the corrector to a domain: omega += network(features)/out_scale, projected onto the
 * 1/2-rule disc (Hermitian, zero mean) as Algorithm 1's post-processing does.  scratch: a
 * device buffer of 5*n*n floats. */
ttsh_status ttsh_fno_correct(ttsh_fno* f, ttsh_domain* d, float* scratch);
/* Corrected rollout: nsteps solver steps of the domain with a correction after every
 * correct_every steps (a trailing partial period is stepped without correction).  One
 * period is recorded as a CUDA graph and replayed.  correct_every must be in [1, 64].
 * Synchronises. */
ttsh_status ttsh_fno_rollout(ttsh_fno* f, ttsh_domain* d, int64_t nsteps, int32_t correct_every, float* scratch);

/* Test hook of the failure path (no counterpart in the paper): launches, on the domain's
 * stream, one block whose bounded wait is on an mbarrier phase that nothing completes, limited
 * to `seconds` (0 < seconds <= 1, else TTSH_E_INVALID).  The wait runs out and sets the
 * domain's status word exactly as a lost TMA, bulk-copy or tensor-core completion would, so
 * the next ttsh_synchronize returns TTSH_E_TIMEOUT once; the CUDA context and the domain
 * stay usable.  (Production waits are limited to 2 s.) */
ttsh_status ttsh_test_bounded_wait(ttsh_domain* d, double seconds);

/* Measured arithmetic peak of the current GPU, for roofline reports (no counterpart in the
 * paper): one launch of a probe kernel in which every thread of 8 blocks of 256 per SM runs 8
 * independent fused multiply-add chains for `iters` iterations in the given precision (32 or
 * 64), timed with CUDA events; *tflops = 2 x chains x iters x threads / time.  iters in
 * [1, 2^24] (TTSH_E_INVALID otherwise).  Synchronises its own stream; allocates 8 bytes. */
ttsh_status ttsh_fma_peak(int32_t precision, int32_t iters, double* tflops);

/* Block the host until the domain's stream is idle; reports deferred CUDA errors, and
 * TTSH_E_TIMEOUT (once) if a bounded wait inside a kernel ran out since the last report (the
 * affected steps are not valid; ttsh_diagnostics reports it too). */
ttsh_status ttsh_synchronize(ttsh_domain* d);

/* Steps taken since the last set_velocity / set_spectral_state. */
int64_t ttsh_step_count(const ttsh_domain* d);

/* Message describing the last failure on the calling thread ("" if none). */
const char* ttsh_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TTSH_H */
