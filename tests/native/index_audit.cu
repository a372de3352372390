// Host audit of the index arithmetic of the fused kernels (csrc/pairconv_c64.cuh and
// csrc/pairconv_tma.cuh), for every supported grid side and pencil layout, without a GPU:
// every shared-memory, stage-buffer, pencil-blocked and Tensor Memory index the kernels form
// stays inside its buffer, each stage covers the pair grid exactly once, the X-stage pencil
// permutation is a permutation with the bank property it is built for, and the barriers the
// kernels leave out (x-slab named barriers, warp-local planes) guard only data that the same
// threads wrote.  Built and run by tests/test_index_audit_host.py; prints one line per check
// group and exits non-zero on the first violation.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../../paper_1507_05156_gb300/csrc/pairconv_tma.cuh"

using namespace hse;

static int g_fail = 0;
#define CHECK(cond, ...)                                 \
  do {                                                   \
    if (!(cond)) {                                       \
      std::printf("FAIL n=%d: ", N_);                    \
      std::printf(__VA_ARGS__);                          \
      std::printf("\n");                                 \
      ++g_fail;                                          \
      return;                                            \
    }                                                    \
  } while (0)

// cells x Q + y P + z of the pair grid, marked in a map over GRID_CPX slots
template <int n>
static std::vector<int> cell_map() {
  using G = Geo<n>;
  std::vector<int> m(G::GRID_CPX, -1);
  for (int x = 0; x < n; ++x)
    for (int y = 0; y < n; ++y)
      for (int z = 0; z < n; ++z) m[x * G::Q + y * G::P + z] = (x * n + y) * n + z;
  return m;
}

// Each stage (Z: zs + e, Y: ys + e P, X: xs + e Q) addresses every grid cell exactly once.
template <int n>
static void audit_stages() {
  constexpr int N_ = n;
  using G = Geo<n>;
  const std::vector<int> cells = cell_map<n>();
  int used = 0;
  for (int v : cells) used += v >= 0;
  CHECK(used == G::N, "the pitches P=%d Q=%d alias grid cells", G::P, G::Q);
  for (int stage = 0; stage < 4; ++stage) {  // Z, Y, X, X in the bank-spread order
    std::vector<int> hit(G::GRID_CPX, 0);
    constexpr XPermTable<n> perm = make_xperm<n, n * n>();
    for (int p = 0; p < G::NN; ++p) {
      const Pencil<n> pc(stage == 3 ? (int)perm.v[p] : p);
      for (int e = 0; e < n; ++e) {
        const int a = stage == 0 ? pc.zs + e : stage == 1 ? pc.ys + e * G::P : pc.xs + e * G::Q;
        CHECK(a >= 0 && a < G::GRID_CPX, "stage %d pencil %d element %d: smem index %d outside [0, %d)", stage, p, e,
              a, G::GRID_CPX);
        CHECK(cells[a] >= 0, "stage %d pencil %d element %d: index %d is padding", stage, p, e, a);
        ++hit[a];
      }
      if (stage != 3) CHECK(pc.zg == p * n, "pencil %d: global z-pencil offset %d", p, pc.zg);
    }
    for (int a = 0; a < G::GRID_CPX; ++a)
      CHECK(hit[a] == (cells[a] >= 0 ? 1 : 0), "stage %d: grid slot %d addressed %d times", stage, a, hit[a]);
  }
  std::printf("n=%d stages: Z, Y, X and permuted X each cover the %d cells once (P=%d, Q=%d)\n", n, G::N, G::P, G::Q);
}

// The X-stage permutation: a permutation of the pencils, and every aligned group of 16 in its
// first part takes 16 distinct 8-byte banks (y P + z mod 16).
template <int n>
static void audit_xperm() {
  constexpr int N_ = n;
  using G = Geo<n>;
  constexpr XPermTable<n> perm = make_xperm<n, n * n>();
  std::vector<int> seen(G::NN, 0);
  for (int i = 0; i < G::NN; ++i) {
    CHECK(perm.v[i] < G::NN, "entry %d = %d out of range", i, (int)perm.v[i]);
    ++seen[perm.v[i]];
  }
  for (int p = 0; p < G::NN; ++p) CHECK(seen[p] == 1, "pencil %d appears %d times", p, seen[p]);
  int cnt[16] = {};
  for (int p = 0; p < G::NN; ++p) ++cnt[((p / n) * G::P + p % n) % 16];
  int ming = G::NN;
  for (int r = 0; r < 16; ++r) ming = cnt[r] < ming ? cnt[r] : ming;
  for (int g = 0; g < ming; ++g) {
    int mask = 0;
    for (int l = 0; l < 16; ++l) {
      const int p = perm.v[16 * g + l];
      mask |= 1 << (((p / n) * G::P + p % n) % 16);
    }
    CHECK(mask == 0xFFFF, "half-warp group %d repeats a bank (mask %04x)", g, mask);
  }
  std::printf("n=%d X permutation: a permutation; %d of %d half-warp groups bank-distinct\n", n, ming, G::NN / 16);
}

// Pencil-blocked layout: chunk e of pencil p at float4 (p >> 5) (n/2) 32 + 32 e + (p & 31),
// inside the NBK complex values of a blocked orbital, each once; the relayout kernel writes the
// same position.
template <int n>
static void audit_blocked() {
  constexpr int N_ = n;
  using G = Geo<n>;
  const int h = n / 2;
  const int nbk4 = (int)(OrbBlk<n>::NBK / 2);
  std::vector<int> hit(nbk4, 0);
  for (int p = 0; p < G::NN; ++p)
    for (int e = 0; e < h; ++e) {
      const int off = (p >> 5) * h * 32 + (p & 31) + 32 * e;
      const int copy = ((p >> 5) * h + e) * 32 + (p & 31);
      CHECK(off == copy, "pencil %d chunk %d: kernel %d, relayout %d", p, e, off, copy);
      CHECK(off >= 0 && off < nbk4, "pencil %d chunk %d: float4 %d outside [0, %d)", p, e, off, nbk4);
      ++hit[off];
    }
  int used = 0;
  for (int v : hit) {
    CHECK(v <= 1, "a blocked float4 is used twice");
    used += v;
  }
  CHECK(used == G::N / 2, "blocked layout covers %d of %d float4", used, G::N / 2);
  std::printf("n=%d blocked layout: %d float4 of %d, each once\n", n, used, nbk4);
}

// A pencil-load layout (PPT passes of TS threads per owner slot): its passes cover the
// pencils once, whole warps, and its TMEM columns fit the allocation.
template <int n, int PPT, int TS>
static void audit_pencil_layout() {
  constexpr int N_ = n;
  using G = Geo<n>;
  using GP = GeoP<n, PPT, TS>;
  std::vector<int> hit(G::NN, 0);
  for (int t = 0; t < TS; ++t)
    for (int ps = 0; ps < PPT; ++ps) {
      if (TS * PPT != G::NN && t + ps * TS >= G::NN) break;
      ++hit[t + ps * TS];
    }
  for (int p = 0; p < G::NN; ++p) CHECK(hit[p] == 1, "PPT=%d TS=%d: pencil %d taken %d times", PPT, TS, p, hit[p]);
  CHECK(GP::THREADS % 32 == 0 && GP::THREADS >= G::T * TS, "PPT=%d TS=%d: %d threads", PPT, TS, GP::THREADS);
  CHECK((G::NN - (PPT - 1) * TS) % 32 == 0 || PPT * TS == G::NN, "PPT=%d TS=%d: ragged pass not whole warps", PPT,
        TS);
  for (int w = 0; w < GP::WARPS; ++w) {
    const int first = (w >> 2) * GP::COLS_PER_WARP;
    CHECK(first + GP::COLS_PER_WARP <= GP::TMEM_COLS && GP::TMEM_COLS <= 512,
          "PPT=%d TS=%d: warp %d columns [%d, %d) beyond %d", PPT, TS, w, first, first + GP::COLS_PER_WARP,
          GP::TMEM_COLS);
  }
  // every kernel row / accumulator row of a thread stays in its warp's columns
  CHECK(GP::TAB + PPT * n <= GP::COLS_PER_WARP && PPT * G::ROW <= GP::TAB, "PPT=%d TS=%d: row layout", PPT, TS);
  // x-slab named barriers: what a slab group's Y stage reads its own Z stage wrote, and what
  // its Z inverse reads its own Y inverse wrote
  constexpr int SB = slab_bar_threads<n, PPT, TS>();
  if constexpr (SB > 0) {
    CHECK(SB % 32 == 0 && G::NN % SB == 0 && G::NN / SB <= 15, "slab groups of %d threads", SB);
    std::vector<int> owner(G::GRID_CPX, -1);
    for (int p = 0; p < G::NN; ++p)
      for (int e = 0; e < n; ++e) owner[Pencil<n>(p).zs + e] = p / SB;  // Z: thread p = pencil p
    for (int p = 0; p < G::NN; ++p)
      for (int e = 0; e < n; ++e)
        CHECK(owner[Pencil<n>(p).ys + e * G::P] == p / SB, "slab group %d reads a cell of group %d", p / SB,
              owner[Pencil<n>(p).ys + e * G::P]);
    std::printf("n=%d PPT=%d TS=%d: %d slab groups of %d threads are closed under Z <-> Y\n", n, PPT, TS,
                G::NN / SB, SB);
  }
  std::printf("n=%d pencil layout PPT=%d TS=%d: %d threads, TMEM %d columns\n", n, PPT, TS, GP::THREADS, GP::TMEM_COLS);
}

// A staged-partner layout: stage rows and pitches, TMA alignment, TMEM, warp-local planes.
template <int n, template <int> class L>
static void audit_staged_layout() {
  constexpr int N_ = n;
  using G = Geo<n>;
  using Lay = L<n>;
  using S = GeoS<n, Lay>;
  if constexpr (!S::FITS) {
    std::printf("n=%d staged layout PPT=%d: not built (does not fit)\n", n, Lay::PPT);
    return;
  } else {
    CHECK(S::STAGE_ROWS >= G::NN, "stage rows %d < %d pencils", S::STAGE_ROWS, G::NN);
    CHECK((S::SP * 8) % 16 == 0 && S::SP >= n, "stage pitch %d complex", S::SP);
    CHECK((S::BR * S::SP * 8) % 16 == 0, "a box of %d rows is not a whole number of 16-byte units", S::BR);
    for (int p = 0; p < G::NN; ++p) {
      const int base = (Pencil<n>(p).zg / n) * S::SP;
      CHECK(base + n <= S::STAGE_CPX, "pencil %d reads stage [%d, %d) beyond %d", p, base, base + n, S::STAGE_CPX);
    }
    CHECK(S::TMEM_COLS <= 512, "TMEM %d columns", S::TMEM_COLS);
    for (int w = 0; w < Lay::WARPS; ++w)
      CHECK((w >> 2) * Lay::COLS_PER_WARP + Lay::COLS_PER_WARP <= S::TMEM_COLS, "warp %d TMEM columns", w);
    if constexpr (Lay::GROUPED) {
      // warp-local planes: the Y stage of a warp reads only cells its own Z stage wrote
      // (thread t of the block serves owner slot t / TS, whose grid starts at slot GRID_CPX)
      std::vector<int> owner((size_t)G::T * G::GRID_CPX, -1);
      for (int t = 0; t < G::T * Lay::TS; ++t) {
        const int slot = t / Lay::TS, tt = t - slot * Lay::TS;
        for (int ps = 0; ps < Lay::PPT; ++ps)
          for (int e = 0; e < n; ++e) owner[slot * G::GRID_CPX + Pencil<n>(tt + ps * Lay::TS).zs + e] = t / 32;
      }
      for (int t = 0; t < G::T * Lay::TS; ++t) {
        const int slot = t / Lay::TS, tt = t - slot * Lay::TS;
        for (int ps = 0; ps < Lay::PPT; ++ps)
          for (int e = 0; e < n; ++e) {
            const int a = slot * G::GRID_CPX + Pencil<n>(tt + ps * Lay::TS).ys + e * G::P;
            CHECK(owner[a] == t / 32, "warp %d's Y stage reads a cell written by warp %d", t / 32, owner[a]);
          }
      }
    }
    std::printf("n=%d staged layout PPT=%d: %d threads, stage %d rows x pitch %d, TMEM %d columns%s\n", n, Lay::PPT,
                Lay::THREADS, S::STAGE_ROWS, S::SP, S::TMEM_COLS, Lay::GROUPED ? ", warp-local planes" : "");
  }
}

template <int n>
static void audit_side() {
  audit_stages<n>();
  audit_xperm<n>();
  audit_blocked<n>();
  audit_pencil_layout<n, 2, Geo<n>::NN / 2>();
  if constexpr (Geo<n>::NN % 32 == 0 && Geo<n>::NN <= 1024 && Geo<n>::T == 1 && n % 4 == 0) audit_pencil_layout<n, 1, Geo<n>::NN>();
  if constexpr (n == 24) audit_pencil_layout<n, 2, 384>();
  audit_staged_layout<n, LayoutSeq>();
  audit_staged_layout<n, LayoutOne>();
}

int main() {
  audit_side<4>();
  audit_side<6>();
  audit_side<8>();
  audit_side<10>();
  audit_side<12>();
  audit_side<16>();
  audit_side<18>();
  audit_side<20>();
  audit_side<24>();
  std::printf(g_fail ? "index audit FAILED (%d)\n" : "index audit ok\n", g_fail);
  return g_fail ? 1 : 0;
}
