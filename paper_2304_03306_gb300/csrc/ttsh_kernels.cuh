// ttsh_kernels.cuh - sm_103a kernels of the confined TTSH solver (templated on precision T
// and grid size N).
//
// One step of Algorithm 1 (Appendix D) is two fused kernels:
//
//   row pass  (one block per R rows of the N x N box, real space)
//     inverse row transforms of omega^, i kx omega^, i ky omega^, v^x, v^y (column-
//     transformed by the previous column pass), giving omega, d_x omega, d_y omega, v_x,
//     v_y (line 2's iDFT[i k omega^] and the ENSURE'd v);
//     rhs1 = -b |v|^2 v - gamma_v K v, rhs2 = -lambda v.grad(omega) - gamma_w K omega
//     (lines 1-2); forward row transforms of the three rhs fields, keeping only the
//     columns mx <= N/4 that the 1/2 rule can keep.
//
//   column pass (one block per stored column mx = 0..N/4, Fourier space)
//     forward column transforms of the three rhs fields; curl assembly
//     rhs^ = i(kx R^1y - ky R^1x) + R^2 (line 3); integrating-factor Euler update (line 4);
//     k = 0: omega^ = 0 and v^(0) <- exp((a-1) dt)(v^(0) + dt R^1(0)) (lines 6-8, Eq. avg);
//     zero |m|^2 > (N/4)^2 (lines 9-11); Hermitian average (line 13, only the mx = 0
//     column needs it in half-spectrum storage); then psi^ = omega^/k^2 and v^ =
//     (i ky psi^, -i kx psi^) (lines 14-15) and the inverse column transforms of the four
//     fields the next row pass needs.
//
// Inter-pass buffers are column-major, [field][mx][y], so the column pass streams whole
// columns and the row pass reads/writes R consecutive y per column.
#pragma once

#include "ttsh_fft.cuh"

namespace ttsh {

// ---------------------------------------------------------------------------------------
// Arguments (all device pointers belong to one domain's workspace)
// ---------------------------------------------------------------------------------------
template <typename T>
struct Args {
  cplx<T>* what;        // state omega^, [mx][j], H x NK
  T* vmean;             // v^(0), 2 values
  T* K;                 // processed mask, N x N
  cplx<T>* G;           // column-pass output / row-pass input, [4][H][N]
  cplx<T>* Rr;          // row-pass output / column-pass input, [3][H][N]
  const cplx<T>* tw;    // W_N^m, m in [0, N)
  double* real;         // double staging, [3][N][N]
  double* part;         // per-block diagnostic partial sums
  T a, b, lam, gv, gw, dt, dk, mean_decay;   // mean_decay = exp((a - 1) dt)
  double dx, cx, cy;    // grid spacing and the psi centre
};

enum RowKind { ROW_STEP = 0, ROW_FWD_VEL = 1, ROW_FWD_MASK = 2, ROW_INV_FIELDS = 3,
               ROW_INV_MASK = 4, ROW_INV_DIAG = 5 };
enum ColMode { COL_STEP = 0, COL_PROLOGUE = 1, COL_PROJECT = 2, COL_MASK = 3 };

constexpr int kDiagQ = 5;   // per-block partials: sum|v|^2, sum w^2, sum|e_th.v|, sum|v|, #nonfinite

// Points per thread of the register butterflies.
template <typename T>
__host__ __device__ constexpr int points_per_thread() { return sizeof(T) == 4 ? 16 : 8; }

template <int KIND> __host__ __device__ constexpr int row_inv_fields() {
  return KIND == ROW_STEP ? 5 : KIND == ROW_INV_FIELDS ? 3 : KIND == ROW_INV_DIAG ? 3
       : KIND == ROW_INV_MASK ? 1 : 0;
}
template <int KIND> __host__ __device__ constexpr int row_fwd_fields() {
  return KIND == ROW_STEP ? 3 : KIND == ROW_FWD_VEL ? 2 : KIND == ROW_FWD_MASK ? 1 : 0;
}
template <int KIND> __host__ __device__ constexpr int row_max_fields() {
  return cmax(row_inv_fields<KIND>(), row_fwd_fields<KIND>());
}

// Row-pass geometry: R rows per block, NT threads.
template <typename T, int N, int KIND>
struct RowCfg {
  static constexpr int L = N / 2;
  static constexpr int PE = cmin(points_per_thread<T>(), L);
  static constexpr int PS = ilog2(PE);
  static constexpr int LP = padded_len<L, PS>();
  static constexpr int TT = L / PE;
  static constexpr int F = row_max_fields<KIND>();
  static constexpr int bytes_per_row = F * LP * (int)sizeof(cplx<T>);
  // Rows per block: up to 32 bytes of consecutive y per column segment (4 floats / 2
  // doubles complex), fewer if the shared memory would exceed ~110 KB.
  static constexpr int R0 = sizeof(T) == 4 ? 4 : 2;
  static constexpr int R = (bytes_per_row * R0 <= 112 * 1024) ? R0
                         : (bytes_per_row * (R0 / 2) <= 112 * 1024 && R0 > 1) ? R0 / 2 : 1;
  static constexpr int NT = cmax(64, cmin(1024, cmax(1, F * R) * TT));
  static constexpr int SMEM = bytes_per_row * R + kDiagQ * 1024 * 8 * (KIND == ROW_INV_DIAG);
};

// Column-pass geometry: FB transforms in flight, NT threads.
template <typename T, int N, int MODE>
struct ColCfg {
  static constexpr int M = N / 4;
  static constexpr int H = M + 1;
  static constexpr int NK = 2 * M + 1;
  static constexpr int PE = cmin(points_per_thread<T>(), N);
  static constexpr int PS = ilog2(PE);
  static constexpr int LP = padded_len<N, PS>();
  static constexpr int TT = N / PE;
  static constexpr int FB0 = MODE == COL_MASK ? 1 : 4;
  static constexpr int FB = (FB0 * LP * (int)sizeof(cplx<T>) <= 160 * 1024) ? FB0
                          : (2 * LP * (int)sizeof(cplx<T>) <= 160 * 1024 && FB0 >= 2) ? 2 : 1;
  static constexpr int NT = cmax(64, cmin(1024, FB * TT));
  static constexpr int SMEM = FB * LP * (int)sizeof(cplx<T>) + NK * (int)sizeof(cplx<T>) + 64;
};

template <typename T>
__device__ __forceinline__ bool finite_t(T v) { return isfinite(v); }

// ---------------------------------------------------------------------------------------
// Row kernels
// ---------------------------------------------------------------------------------------
template <typename T, int N, int KIND>
__global__ void __launch_bounds__(RowCfg<T, N, KIND>::NT)
row_kernel(Args<T> A) {
  using Cfg = RowCfg<T, N, KIND>;
  constexpr int L = Cfg::L, M = N / 4, H = M + 1;
  constexpr int R = Cfg::R, NT = Cfg::NT, PE = Cfg::PE, PS = Cfg::PS, LP = Cfg::LP;
  constexpr int FI = row_inv_fields<KIND>();
  constexpr int FF = row_fwd_fields<KIND>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* sm = reinterpret_cast<cplx<T>*>(smem_raw);
  const int y0 = blockIdx.x * R;
  const int tid = threadIdx.x;
  const cplx<T>* __restrict__ tw = A.tw;

  // ---- inverse row transforms (C2R through an L-point complex transform) ----
  if constexpr (FI > 0) {
    for (int e = tid; e < FI * R * L; e += NT) {
      const int r = e % R;
      const int t = e / R;
      const int k = t % L;
      const int f = t / L;
      // spectral source of field f: which G plane and whether to multiply by i kx
      int plane;
      bool dx_mul = false;
      if constexpr (KIND == ROW_STEP) {
        plane = f == 0 ? 0 : f == 1 ? 0 : f - 1;   // w, i kx w, (i ky w), vx, vy
        dx_mul = (f == 1);
      } else if constexpr (KIND == ROW_INV_MASK) {
        plane = 0;
      } else {
        plane = f == 0 ? 0 : f + 1;                 // w, vx, vy
      }
      const cplx<T>* src = A.G + (size_t)plane * H * N + (y0 + r);
      cplx<T> X = mk<T>(0, 0), Xm = mk<T>(0, 0);
      if (k <= M) X = src[(size_t)k * N];
      const int km = L - k;
      if (km <= M) Xm = src[(size_t)km * N];
      if (dx_mul) {
        X = mul_i(X) * (A.dk * (T)k);
        Xm = mul_i(Xm) * (A.dk * (T)km);
      }
      if (k == 0) X.y = 0;   // the mx = 0 entry of a real row is real
      const cplx<T> w = conjg(tw[k]);          // conj(W_N^k)
      const cplx<T> s = X + conjg(Xm);
      const cplx<T> d = X - conjg(Xm);
      sm[(f * R + r) * LP + padi<PS>(k)] = s + mul_i(cmul(w, d));
    }
    fft_batch<T, L, PE, +1, NT, N>(sm, FI * R, tw);
  }

  // ---- real-space work ----
  // element x of a real row lives in complex slot x/2 (re for even x, im for odd x)
  auto rl = [&](int f, int r, int x) -> T& {
    cplx<T>& c = sm[(f * R + r) * LP + padi<PS>(x >> 1)];
    return (x & 1) ? c.y : c.x;
  };

  if constexpr (KIND == ROW_STEP) {
    for (int e = tid; e < R * N; e += NT) {
      const int r = e / N, x = e % N;
      const T w = rl(0, r, x), wx = rl(1, r, x), wy = rl(2, r, x);
      const T vx = rl(3, r, x), vy = rl(4, r, x);
      const T Kv = A.K[(size_t)(y0 + r) * N + x];
      const T v2 = vx * vx + vy * vy;
      const T c1 = -A.b * v2 - A.gv * Kv;               // line 1
      rl(0, r, x) = c1 * vx;
      rl(1, r, x) = c1 * vy;
      rl(2, r, x) = -A.lam * (vx * wx + vy * wy) - A.gw * Kv * w;   // line 2
    }
  } else if constexpr (KIND == ROW_FWD_VEL || KIND == ROW_FWD_MASK) {
    __syncthreads();
    for (int e = tid; e < FF * R * N; e += NT) {
      const int x = e % N;
      const int t = e / N;
      const int r = t % R, f = t / R;
      rl(f, r, x) = (T)A.real[((size_t)f * N + (y0 + r)) * N + x];
    }
  } else if constexpr (KIND == ROW_INV_FIELDS) {
    for (int e = tid; e < 3 * R * N; e += NT) {
      const int x = e % N;
      const int t = e / N;
      const int r = t % R, f = t / R;
      A.real[((size_t)f * N + (y0 + r)) * N + x] = (double)rl(f, r, x);
    }
  } else if constexpr (KIND == ROW_INV_MASK) {
    for (int e = tid; e < R * N; e += NT) {
      const int r = e / N, x = e % N;
      const T k = rl(0, r, x);
      A.K[(size_t)(y0 + r) * N + x] = k * k;          // K = (iDFT[...])^2
    }
  } else if constexpr (KIND == ROW_INV_DIAG) {
    double acc[kDiagQ] = {0, 0, 0, 0, 0};
    for (int e = tid; e < R * N; e += NT) {
      const int r = e / N, x = e % N;
      const double w = (double)rl(0, r, x);
      const double vx = (double)rl(1, r, x), vy = (double)rl(2, r, x);
      const double px = (x - N / 2) * A.dx - A.cx;
      const double py = (y0 + r - N / 2) * A.dx - A.cy;
      const double rr = sqrt(px * px + py * py);
      const double vn = sqrt(vx * vx + vy * vy);
      acc[0] += vx * vx + vy * vy;
      acc[1] += w * w;
      acc[2] += rr > 0 ? fabs(-py * vx + px * vy) / rr : 0.0;
      acc[3] += vn;
      acc[4] += (isfinite(w) && isfinite(vx) && isfinite(vy)) ? 0.0 : 1.0;
    }
    // fixed-order block reduction (deterministic)
    __syncthreads();
    double* red = reinterpret_cast<double*>(smem_raw + Cfg::bytes_per_row * R);
    for (int q = 0; q < kDiagQ; ++q) red[q * 1024 + tid] = acc[q];
    __syncthreads();
    for (int s = 512; s >= 1; s >>= 1) {
      if (tid < s && tid + s < NT)
        for (int q = 0; q < kDiagQ; ++q) red[q * 1024 + tid] += red[q * 1024 + tid + s];
      __syncthreads();
    }
    if (tid < kDiagQ) A.part[(size_t)blockIdx.x * kDiagQ + tid] = red[tid * 1024];
  }

  // ---- forward row transforms (R2C), keep mx <= N/4 ----
  if constexpr (FF > 0) {
    fft_batch<T, L, PE, -1, NT, N>(sm, FF * R, tw);
    for (int e = tid; e < FF * R * H; e += NT) {
      const int r = e % R;
      const int t = e / R;
      const int k = t % H;
      const int f = t / H;
      const cplx<T>* row = sm + (f * R + r) * LP;
      const cplx<T> Zk = row[padi<PS>(k)];
      const cplx<T> Zm = conjg(row[padi<PS>((L - k) & (L - 1))]);
      const cplx<T> s = Zk + Zm;
      const cplx<T> d = Zk - Zm;
      // X[k] = (Zk + Zm)/2 - (i/2) W^k (Zk - Zm)
      const cplx<T> X = (s - mul_i(cmul(tw[k], d))) * (T)0.5;
      A.Rr[((size_t)f * H + k) * N + (y0 + r)] = X;
    }
  }
}

// ---------------------------------------------------------------------------------------
// Column kernel
// ---------------------------------------------------------------------------------------
template <typename T, int N, int MODE>
__global__ void __launch_bounds__(ColCfg<T, N, MODE>::NT)
col_kernel(Args<T> A) {
  using Cfg = ColCfg<T, N, MODE>;
  constexpr int M = N / 4, H = M + 1, NK = 2 * M + 1;
  constexpr int PE = Cfg::PE, PS = Cfg::PS, LP = Cfg::LP, NT = Cfg::NT, FB = Cfg::FB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<T>* buf = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* acc = buf + FB * LP;
  T* s0 = reinterpret_cast<T*>(acc + NK);   // [0..1]: k = 0 forward values, [2..3]: v^(0)
  const int kx = blockIdx.x;
  const int tid = threadIdx.x;
  const T kxp = A.dk * (T)kx;
  const T invN = (T)1 / (T)N;
  const cplx<T>* __restrict__ tw = A.tw;

  auto ky_of = [](int j) { return j <= M ? j : j - NK; };

  // ---- forward column transforms and curl assembly ----
  if constexpr (MODE != COL_PROLOGUE) {
    constexpr int NF = MODE == COL_STEP ? 3 : MODE == COL_PROJECT ? 2 : 1;
    for (int f0 = 0; f0 < NF; f0 += FB) {
      const int nb = cmin(FB, NF - f0);
      for (int e = tid; e < nb * N; e += NT) {
        const int b = e / N, y = e % N;
        buf[b * LP + padi<PS>(y)] = A.Rr[((size_t)(f0 + b) * H + kx) * N + y];
      }
      fft_batch<T, N, PE, -1, NT, N>(buf, nb, tw);
      for (int j = tid; j < NK; j += NT) {
        const int ky = ky_of(j);
        const int idx = ky & (N - 1);
        const T kyp = A.dk * (T)ky;
        cplx<T> a = f0 == 0 ? mk<T>(0, 0) : acc[j];
        for (int b = 0; b < nb; ++b) {
          const int f = f0 + b;
          const cplx<T> v = buf[b * LP + padi<PS>(idx)];
          if constexpr (MODE == COL_MASK) {
            a = v;
          } else {
            // f = 0: (rhs1_x | v_x) -> -i ky; f = 1: (rhs1_y | v_y) -> +i kx; f = 2: rhs2 -> 1
            if (f == 0) a = a - mul_i(v) * kyp;
            else if (f == 1) a = a + mul_i(v) * kxp;
            else a = a + v;
            if (kx == 0 && j == 0 && f < 2) s0[f] = v.x;   // raw k = 0 value (real)
          }
        }
        acc[j] = a;
      }
      __syncthreads();   // buf is refilled by the next batch
    }

    // ---- update (Algorithm 1 lines 3-11) ----
    for (int j = tid; j < NK; j += NT) {
      const int ky = ky_of(j);
      const int m2 = kx * kx + ky * ky;
      cplx<T> wn;
      if constexpr (MODE == COL_STEP) {
        const T k2 = A.dk * A.dk * (T)m2;
        const T om = (T)1 - k2;
        const T E = exp((A.a - om * om) * A.dt);
        const cplx<T> w = A.what[(size_t)kx * NK + j];
        const cplx<T> r = acc[j] * invN;
        wn = (w + r * A.dt) * E;
        if (m2 == 0 || m2 > M * M) wn = mk<T>(0, 0);
      } else if constexpr (MODE == COL_PROJECT) {
        wn = acc[j] * invN;
        if (m2 == 0 || m2 > M * M) wn = mk<T>(0, 0);
      } else {   // COL_MASK: keep |m|^2 <= (N/8)^2, fold both 1/N factors of the round trip
        wn = acc[j] * (invN * invN);
        if (m2 > (N / 8) * (N / 8)) wn = mk<T>(0, 0);
      }
      acc[j] = wn;
    }
    if constexpr (MODE == COL_STEP || MODE == COL_PROJECT) {
      if (kx == 0 && tid == 0) {
        for (int c = 0; c < 2; ++c) {
          T vm;
          if constexpr (MODE == COL_STEP)
            vm = A.mean_decay * (A.vmean[c] + A.dt * (s0[c] * invN));   // line 8
          else
            vm = s0[c] * invN;                                              // DFT[v](0)
          s0[2 + c] = vm;
          A.vmean[c] = vm;
        }
      }
    }
    __syncthreads();
    if constexpr (MODE == COL_STEP || MODE == COL_PROJECT) {
      // line 13: Hermitian average; with half-spectrum storage only mx = 0 pairs are stored
      if (kx == 0) {
        for (int ky = 1 + tid; ky <= M; ky += NT) {
          const cplx<T> p = acc[ky], q = acc[NK - ky];
          const cplx<T> h = (p + conjg(q)) * (T)0.5;
          acc[ky] = h;
          acc[NK - ky] = conjg(h);
        }
        __syncthreads();
      }
      for (int j = tid; j < NK; j += NT) A.what[(size_t)kx * NK + j] = acc[j];
    }
  } else {
    for (int j = tid; j < NK; j += NT) acc[j] = A.what[(size_t)kx * NK + j];
    if (kx == 0 && tid == 0) {
      s0[2] = A.vmean[0];
      s0[3] = A.vmean[1];
    }
    __syncthreads();
  }

  // ---- inverse column transforms of the fields the next row pass reads ----
  constexpr int NI = MODE == COL_MASK ? 1 : 4;
  for (int f0 = 0; f0 < NI; f0 += FB) {
    const int nb = cmin(FB, NI - f0);
    for (int e = tid; e < nb * N; e += NT) {
      const int b = e / N, idx = e % N;
      const int f = f0 + b;
      const int ky = idx <= N / 2 ? idx : idx - N;
      cplx<T> v = mk<T>(0, 0);
      if (ky >= -M && ky <= M) {
        const cplx<T> w = acc[ky >= 0 ? ky : ky + NK];
        if constexpr (MODE == COL_MASK) {
          v = w;
        } else {
          const T kyp = A.dk * (T)ky;
          const int m2 = kx * kx + ky * ky;
          const T k2 = A.dk * A.dk * (T)m2;
          const T inv = m2 > 0 ? invN / k2 : (T)0;
          if (f == 0) v = w * invN;                       // omega
          else if (f == 1) v = mul_i(w) * (kyp * invN);   // i ky omega^ -> d_y omega
          else if (f == 2) v = mul_i(w) * (kyp * inv);    // v^x = i ky psi^   (line 15)
          else v = mul_i(w) * (-kxp * inv);               // v^y = -i kx psi^
          if (m2 == 0 && f >= 2) v = mk<T>(s0[2 + (f - 2)] * invN, (T)0);   // mean flow
        }
      }
      buf[b * LP + padi<PS>(idx)] = v;
    }
    fft_batch<T, N, PE, +1, NT, N>(buf, nb, tw);
    for (int e = tid; e < nb * N; e += NT) {
      const int b = e / N, y = e % N;
      A.G[((size_t)(f0 + b) * H + kx) * N + y] = buf[b * LP + padi<PS>(y)];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// Diagnostics reductions (fixed order, double precision)
// ---------------------------------------------------------------------------------------
// Sum nblocks x kDiagQ partials into out[kDiagQ] with one block of 256 threads.
__global__ void diag_reduce_kernel(const double* __restrict__ part, int nblocks, double* out);

// Per-column shell spectrum: one thread per stored column, sequential over its modes.
template <typename T, int N>
__global__ void spectrum_col_kernel(Args<T> A, int nbins, double* __restrict__ colhist,
                                    int* __restrict__ badcount) {
  constexpr int M = N / 4, H = M + 1, NK = 2 * M + 1;
  const int kx = blockIdx.x * blockDim.x + threadIdx.x;
  if (kx >= H) return;
  double* h = colhist + (size_t)kx * nbins;
  for (int s = 0; s < nbins; ++s) h[s] = 0.0;
  const double dk = (double)A.dk;
  const double wgt = kx > 0 ? 2.0 : 1.0;   // mx > 0 columns stand for +-mx
  int bad = 0;
  for (int j = 0; j < NK; ++j) {
    const int ky = j <= M ? j : j - NK;
    const int m2 = kx * kx + ky * ky;
    const cplx<T> w = A.what[(size_t)kx * NK + j];
    const double wr = (double)w.x, wi = (double)w.y;
    if (!isfinite(wr) || !isfinite(wi)) ++bad;
    double e;
    if (m2 == 0) {
      const double u = (double)A.vmean[0], v = (double)A.vmean[1];
      e = u * u + v * v;
    } else {
      e = (wr * wr + wi * wi) / (dk * dk * (double)m2);
    }
    const int s = (int)rint(sqrt((double)m2));
    if (s < nbins) h[s] += wgt * e;
  }
  if (bad) atomicAdd(badcount, bad);
}

__global__ void spectrum_reduce_kernel(const double* __restrict__ colhist, int ncols, int nbins,
                                       double scale, double* __restrict__ out);

}  // namespace ttsh
