// Host-side index checks of the step kernels' shared-memory plans and index maps, for every
// tile variant the library registers (the lists below mirror the variant tables of
// csrc/ttsh_ops_impl.cuh).  Compiled and run by tests/test_geometry.py; no GPU is needed:
// every quantity here is a compile-time constant of the kernel headers or an index the
// kernels compute from them, replayed on the CPU.
//
// Checked, for each variant:
//   - the Stockham transforms of the row (length N/2) and column (length N) passes: every
//     stage reads each element once and writes each once, inside the padded buffer; where a
//     stage addresses a thread's accesses as compile-time offsets from one padded base, the
//     offsets equal the padded indices; per-stage twiddle-table entries stay in the table;
//   - the row pass's shared-memory regions: aligned, disjoint, inside the launch's bytes;
//   - the row pass's G-tile staging: every copy aligned to its size and inside its plane,
//     every source chunk inside its column's rows of G; every slot the first inverse stage
//     reads was written by the staging (of this block, or of the other block of a cluster);
//   - the column pass's regions and its staging copies and reads.
#include <cstdio>
#include <vector>

#include "ttsh_kernels.cuh"

using namespace ttsh;

static int g_fail = 0, g_checked = 0;

// Shared memory a one-block-per-SM launch with programmatic dependent launch reserves per
// block (kSpreadSmem of the launchers in csrc/ttsh_ops_impl.cuh): every pass must still fit
// with its static shared memory on top.
static constexpr int kSpreadSmemBytes = 116 * 1024;

#define CHECK(c, ...)                                                \
  do {                                                               \
    if (!(c)) {                                                      \
      if (++g_fail <= 40) {                                          \
        std::printf("FAIL line %d: %s | ", __LINE__, #c);            \
        std::printf(__VA_ARGS__);                                    \
        std::printf("\n");                                           \
      }                                                              \
    }                                                                \
  } while (0)

// padded index: one spare slot after every 2^ps slots
static constexpr int padded(int i, int ps) { return i + (i >> ps); }
// the rotated layout of one stage handoff with 4 or 8 points per thread (see stockham_stage)
static constexpr int rotated(int i, int pe) {
  return pe == 4 ? (i & ~15) | ((i + ((i >> 2) & 12)) & 15) : (i & ~15) | ((i + ((i >> 3) & 8)) & 15);
}

template <typename T>
static const char* tname() { return sizeof(T) == 4 ? "f32" : "f64"; }

// ------------------------------------------------------------------ transforms
template <typename T, int L, int PE>
static void check_fft(const char* who) {
  constexpr int PS = pad_shift<T>();
  constexpr int LP = padded_len<L, PS>();
  constexpr int TT = L / PE;
  constexpr bool kStageTab = StageTab<T, L, PE>::USE;
  constexpr int kStageEntries = StageTab<T, L, PE>::ENTRIES;
  static_assert(L % PE == 0, "points per thread must divide the length");
  // slot in which the previous stage stored each element (the input layout is padded)
  std::vector<int> handed(L);
  for (int i = 0; i < L; ++i) handed[i] = padded(i, PS);
  for (int Ns = 1; Ns < L;) {
    const int R = (L / Ns < PE) ? (L / Ns) : PE;
    const int SL = L / R, NB = PE / R;
    const bool ld_off = SL % (1 << PS) == 0 || L <= (1 << PS);
    const bool st_off = Ns % (1 << PS) == 0 || Ns * R <= (1 << PS);
    const bool rotate = PE == 4 || (PE == 8 && sizeof(T) == 4);
    const bool rot_out = rotate && Ns == PE && R == PE && Ns * R < L;
    const bool rot_in = rotate && Ns == PE * PE && L > PE * PE;
    std::vector<int> rd(L, 0), wr(L, 0), rslot(LP, 0), wslot(LP, 0), next(L, -1);
    for (int j = 0; j < TT; ++j)
      for (int b = 0; b < NB; ++b) {
        const int q = j + b * TT;
        const int k = q & (Ns - 1);
        const int base = (q - k) * R + k;
        for (int r = 0; r < R; ++r) {
          const int li = q + r * SL, si = base + r * Ns;
          CHECK(li >= 0 && li < L && si >= 0 && si < L, "%s L=%d PE=%d Ns=%d", who, L, PE, Ns);
          if (li < 0 || li >= L || si < 0 || si >= L) continue;
          ++rd[li];
          ++wr[si];
          const int lslot = rot_in ? rotated(li, PE) : padded(li, PS);
          const int sslot = rot_out ? rotated(si, PE) : padded(si, PS);
          CHECK(lslot >= 0 && lslot < LP && sslot >= 0 && sslot < LP, "%s L=%d Ns=%d", who, L, Ns);
          if (lslot < 0 || lslot >= LP || sslot < 0 || sslot >= LP) continue;
          ++rslot[lslot];
          ++wslot[sslot];
          CHECK(lslot == handed[li], "%s L=%d Ns=%d: element %d loaded from another slot than stored", who, L, Ns, li);
          next[si] = sslot;
          if (ld_off && !rot_in)
            CHECK(padded(li, PS) == padded(q, PS) + r * SL + ((r * SL) >> PS), "%s L=%d Ns=%d q=%d r=%d", who, L, Ns, q, r);
          if (st_off && !rot_out)
            CHECK(padded(si, PS) == padded(base, PS) + r * Ns + ((r * Ns) >> PS), "%s L=%d Ns=%d q=%d r=%d", who, L, Ns,
                  q, r);
          if (kStageTab && Ns > 1 && r > 0)
            CHECK(stage_offset(L, PE, Ns) + (r - 1) * Ns + k < kStageEntries, "%s L=%d Ns=%d", who, L, Ns);
        }
      }
    for (int i = 0; i < L; ++i) CHECK(rd[i] == 1 && wr[i] == 1, "%s L=%d PE=%d Ns=%d i=%d", who, L, PE, Ns, i);
    for (int i = 0; i < LP; ++i) CHECK(rslot[i] <= 1 && wslot[i] <= 1, "%s L=%d PE=%d Ns=%d slot=%d", who, L, PE, Ns, i);
    // the layout a stage stores is the one the next stage loads
    if (rot_out) CHECK(Ns * R == PE * PE, "%s L=%d: rotated output not read by the Ns = PE^2 stage", who, L);
    handed = next;
    Ns *= R;
  }
  // callers read the result in the padded layout
  for (int i = 0; i < L; ++i) CHECK(handed[i] == padded(i, PS), "%s L=%d: output %d not in the padded layout", who, L, i);
}

// ------------------------------------------------------------------ row pass
template <typename T, int N, int KIND, int R, int PEV, int CL = 1, int CMP = 0>
static void check_row() {
  using G = RowGeo<T, N, KIND, R, PEV, CL, CMP>;
  if constexpr (G::VALID) {
    ++g_checked;
    char who[96];
    std::snprintf(who, sizeof who, "row %s N=%d kind=%d R=%d PE=%d CL=%d CMP=%d", tname<T>(), N, KIND, R, PEV, CL, CMP);
    constexpr int CB = G::CB;
    check_fft<T, G::L, G::PE>(who);
    // regions
    CHECK(G::OFF_BUF == G::TW_BYTES && G::OFF_BUF % 16 == 0, "%s", who);
    constexpr int kRowLen = padded_len<G::L, G::PS>();
    CHECK((G::F * R - 1) * G::LPR + kRowLen <= G::BUF_BYTES / CB, "%s transform rows", who);
    CHECK(G::OFF_GIN % 128 == 0 && G::OFF_GIN >= G::OFF_BUF + G::BUF_BYTES, "%s", who);
    CHECK(G::OFF_KS % 16 == 0 && G::OFF_KS >= G::OFF_GIN + (G::STAGE_G ? G::GIN_BYTES : 0), "%s", who);
    CHECK(G::OFF_RED % 16 == 0 && G::OFF_RED >= G::OFF_KS + (G::STAGE_K ? G::KS_BYTES : 0), "%s", who);
    CHECK(G::OFF_FWD % 16 == 0 && G::OFF_FWD >= G::OFF_RED + G::RED_BYTES, "%s", who);
    CHECK(G::SMEM >= G::OFF_FWD + (G::SEPARATE ? G::BUF_BYTES : 0) + 128, "%s", who);
    CHECK(cmax(G::SMEM, kSpreadSmemBytes) + kRecSmem <= 227 * 1024, "%s launch bytes", who);
    if constexpr (G::STAGE_K) CHECK(R * N * (int)sizeof(T) % 16 == 0 && R * N * (int)sizeof(T) <= G::KS_BYTES, "%s", who);
    if constexpr (G::TMA_OK) CHECK(G::RSP == R && G::H * R * CB <= G::GPS, "%s TMA box", who);
    if constexpr (G::STAGE_G) {
      constexpr int H = G::H, M = G::M, NPL = G::NPL, GPC = G::GPS / CB;
      constexpr int CPS = G::SEG / G::CHUNK;
      CHECK(G::SEG % G::CHUNK == 0 && G::SEGP % G::CHUNK == 0 && G::RSP >= G::RS, "%s", who);
      std::vector<std::vector<char>> wr(CL, std::vector<char>((size_t)NPL * GPC, 0));
      for (int blk = 0; blk < N / R; ++blk) {
        const int crank = blk % CL;
        const int yc = (blk - crank) * R;
        CHECK(yc >= 0 && yc + G::RS <= N, "%s rows of block %d", who, blk);
        const int cbase = crank * G::HC;
        const int ccnt = cmin(G::HC, H - cbase);
        for (int pl = 0; pl < NPL; ++pl)
          for (int i = 0; i < ccnt * CPS; ++i) {
            const long dst = (long)pl * G::GPS + (long)(i / CPS) * G::SEGP + (long)(i % CPS) * G::CHUNK;
            const long src = (((long)pl * H + cbase) * N + yc) * CB + (long)(i / CPS) * N * CB + (long)(i % CPS) * G::CHUNK;
            CHECK(dst % G::CHUNK == 0 && dst + G::CHUNK <= (long)(pl + 1) * G::GPS, "%s dst %ld", who, dst);
            CHECK(src % G::CHUNK == 0 && src + G::CHUNK <= 3L * H * N * CB, "%s src %ld", who, src);
            CHECK(cbase + i / CPS < H && (i % CPS) * G::CHUNK + G::CHUNK <= G::SEG, "%s chunk %d", who, i);
            if (blk < CL)   // every cluster (every block when CL = 1) stages the same slots
              for (long b = dst; b < dst + G::CHUNK; b += CB) wr[crank][b / CB] = 1;
          }
      }
      for (int f = 0; f < NPL; ++f)
        for (int crank = 0; crank < CL; ++crank)
          for (int r = 0; r < R; ++r)
            for (int k = 0; k <= M; ++k) {
              if constexpr (CL == 1) {
                const int slot = f * GPC + k * G::RSP + r;
                CHECK(slot < NPL * GPC && wr[0][slot], "%s read f=%d k=%d r=%d", who, f, k, r);
              } else {
                const int o = k < G::HC ? 0 : 1;
                const int idx = f * GPC + (k - o * G::HC) * G::RS + crank * R + r;
                CHECK(idx < NPL * GPC && wr[o][idx], "%s cluster read f=%d k=%d r=%d", who, f, k, r);
              }
            }
      if constexpr (CL > 1) {   // results written back into the shares, stored in 16-byte pieces
        for (int crank = 0; crank < CL; ++crank) {
          const int ccnt = cmin(G::HC, H - crank * G::HC);
          for (int f = 0; f < NPL; ++f)
            for (int j = 0; j < ccnt; ++j)
              for (int pz = 0; pz < G::SEG / 16; ++pz)
                CHECK((long)f * G::GPS + (long)j * G::SEG + pz * 16 + 16 <= (long)(f + 1) * G::GPS, "%s store", who);
        }
      }
    }
  }
}

// ------------------------------------------------------------------ column pass
template <typename T, int N, int MODE, int PEV>
static void check_col() {
  using G = ColGeo<T, N, MODE, PEV>;
  if constexpr (G::VALID) {
    ++g_checked;
    char who[96];
    std::snprintf(who, sizeof who, "col %s N=%d mode=%d PE=%d", tname<T>(), N, MODE, PEV);
    constexpr int CB = G::CB, LP = G::LP, PS = G::PS;
    check_fft<T, N, G::PE>(who);
    CHECK(G::OFF_BUF == G::TW_BYTES && G::OFF_BUF % 16 == 0, "%s", who);
    CHECK(G::OFF_ACC % 16 == 0 && G::OFF_ACC >= G::OFF_BUF + G::FB * LP * CB, "%s", who);
    CHECK(G::OFF_WS % 16 == 0 && G::OFF_WS >= G::OFF_ACC + G::NK * CB, "%s", who);
    CHECK(G::OFF_STG % 16 == 0 && G::OFF_STG >= G::OFF_WS + (G::WS_BYTES > 0 ? G::NK * CB : 0), "%s", who);
    CHECK(G::OFF_S0 % 16 == 0 && G::OFF_S0 >= G::OFF_STG + (G::BULK ? G::NF * N * CB : 0), "%s", who);
    CHECK(G::SMEM >= G::OFF_S0 + 4 * (int)sizeof(T), "%s", who);
    CHECK(cmax(G::SMEM, kSpreadSmemBytes) + kRecSmem <= 227 * 1024, "%s launch bytes", who);
    CHECK(G::FB >= 1 && G::NT % G::TT == 0, "%s", who);
    if constexpr (G::BULK) {   // one bulk copy of N values per field: 16-byte aligned, whole 16-byte units
      for (int f = 0; f < G::NF; ++f) {
        CHECK((G::OFF_STG + f * N * CB) % 16 == 0 && (N * CB) % 16 == 0, "%s bulk dst", who);
        for (int kx = 0; kx < G::H; ++kx) CHECK((((long)f * G::H + kx) * N * CB) % 16 == 0, "%s bulk src", who);
      }
    }
    // staged inputs (per value) and the reads of the transformed columns
    for (int b = 0; b < G::FB; ++b)
      for (int y = 0; y < N; ++y) CHECK(b * LP + padded(y, PS) < G::FB * LP, "%s buf b=%d y=%d", who, b, y);
  }
}

// ------------------------------------------------------------------ the registered variants
template <typename T, int N>
static void check_size() {
  // row pass: the step variants of the registry, then the other kinds at their default shape
  check_row<T, N, ROW_STEP, default_step_rows<T, N>(), default_step_row_pe<T, N>(), default_row_cluster<T, N>()>();
  if constexpr (sizeof(T) == 4) {
    check_row<T, N, ROW_STEP, 4, 16>();
    check_row<T, N, ROW_STEP, 2, 16>();
    check_row<T, N, ROW_STEP, 1, 16>();
    check_row<T, N, ROW_STEP, 2, 8>();
    if constexpr (N >= 2048) {
      check_row<T, N, ROW_STEP, 1, 16, 2>();
      check_row<T, N, ROW_STEP, 2, 16, 2>();
    }
    if constexpr (N >= 1024 && N <= 4096) {
      check_row<T, N, ROW_STEP, 2, 16, 1, 1>();
      check_row<T, N, ROW_STEP, 1, 16, 2, 1>();
      check_row<T, N, ROW_STEP, 1, 16, 1, 1>();
    }
  } else {
    check_row<T, N, ROW_STEP, 2, 8>();
    check_row<T, N, ROW_STEP, 1, 8>();
    check_row<T, N, ROW_STEP, 1, 4>();
  }
  check_row<T, N, ROW_FWD_VEL, default_rows<T, N>(), default_row_pe<T, N>()>();
  check_row<T, N, ROW_FWD_MASK, default_rows<T, N>(), default_row_pe<T, N>()>();
  check_row<T, N, ROW_INV_FIELDS, default_rows<T, N>(), default_row_pe<T, N>()>();
  check_row<T, N, ROW_INV_MASK, default_rows<T, N>(), default_row_pe<T, N>()>();
  check_row<T, N, ROW_INV_DIAG, default_rows<T, N>(), default_row_pe<T, N>()>();
  // column pass: the step variants, then the other modes at their default shape
  check_col<T, N, COL_STEP, default_step_col_pe<T, N>()>();
  if constexpr (sizeof(T) == 4) {
    check_col<T, N, COL_STEP, 8>();
    check_col<T, N, COL_STEP, 16>();
    check_col<T, N, COL_STEP, 4>();
  } else {
    check_col<T, N, COL_STEP, 8>();
    check_col<T, N, COL_STEP, 4>();
  }
  check_col<T, N, COL_PROLOGUE, default_col_pe<T, N>()>();
  check_col<T, N, COL_PROJECT, default_col_pe<T, N>()>();
  check_col<T, N, COL_MASK, default_col_pe<T, N>()>();
  check_col<T, N, COL_ADDW, default_col_pe<T, N>()>();
  check_col<T, N, COL_DIV, default_col_pe<T, N>()>();
}

int main() {
  check_size<float, 16>();
  check_size<float, 32>();
  check_size<float, 64>();
  check_size<float, 128>();
  check_size<float, 256>();
  check_size<float, 512>();
  check_size<float, 1024>();
  check_size<float, 2048>();
  check_size<float, 4096>();
  check_size<float, 8192>();
  check_size<double, 16>();
  check_size<double, 32>();
  check_size<double, 64>();
  check_size<double, 128>();
  check_size<double, 256>();
  check_size<double, 512>();
  check_size<double, 1024>();
  check_size<double, 2048>();
  check_size<double, 4096>();
  std::printf("%d pass plans checked, %d failures\n", g_checked, g_fail);
  return g_fail == 0 && g_checked > 0 ? 0 : 1;
}
