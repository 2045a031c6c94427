// Host check of the data-flow strip tables (csrc/sor_strips.cuh): for many
// sizes and warp counts, the strips cover every interior row of every plane
// (cube) or quarter (9-point) and column tile exactly once, carry the numbers
// the kernels decode, keep every access inside the arrays, and list as
// neighbours every strip owning a cell the stencil reaches from theirs
// (brute force over the cells).  Prints the number of failures; exit status
// 0 when there are none.
#include <cstdio>
#include <set>
#include <vector>

#include "sor_strips.cuh"

using namespace sorgb;

static long fails = 0;
#define CHECK(cond, ...)                         \
  do {                                           \
    if (!(cond)) {                               \
      if (fails < 20) std::printf(__VA_ARGS__);  \
      ++fails;                                   \
    }                                            \
  } while (0)

static void check3(int n, int warps) {
  const Layout L = Layout::make(n);
  const int m = n + 2, ct = L.col_tiles();
  std::vector<Tile> s;
  const int bands = build_strips3(L, warps, &s);
  CHECK((long)s.size() == (long)n * bands * ct, "3d n=%d: %zu strips\n", n, s.size());
  std::vector<int> owner((size_t)m * m * ct, -1);
  for (int idx = 0; idx < (int)s.size(); ++idx) {
    const Tile& t = s[idx];
    const int k = t.row0 / m, i0 = t.row0 - k * m, i1 = i0 + t.nrows, tc = (t.col0 - 1) / kWarpCols;
    CHECK(t.col0 == 1 + tc * kWarpCols && tc == idx % ct, "3d n=%d strip %d: column tile\n", n, idx);
    CHECK(k == idx / (bands * ct) + 1, "3d n=%d strip %d: plane %d\n", n, idx, k);
    CHECK(k >= 1 && k <= n && i0 >= 1 && i1 > i0 && i1 <= n + 1, "3d n=%d strip %d: rows\n", n, idx);
    // reads: rows i0-1 .. i1 and planes k-1 .. k+1; columns col0-1 .. col0+128
    CHECK(i0 - 1 >= 0 && i1 <= m - 1 && k - 1 >= 0 && k + 1 <= m - 1, "3d n=%d strip %d: halo rows\n", n, idx);
    CHECK(t.col0 - 1 + kOff >= 0 && t.col0 + kWarpCols + kOff < L.pitch, "3d n=%d strip %d: halo columns\n", n, idx);
    for (int i = i0; i < i1 && i >= 1 && i <= n; ++i) {
      int& o = owner[((size_t)k * m + i) * ct + tc];
      CHECK(o == -1, "3d n=%d: row %d of plane %d tile %d in two strips\n", n, i, k, tc);
      o = idx;
    }
  }
  for (int k = 1; k <= n; ++k)
    for (int i = 1; i <= n; ++i)
      for (int tc = 0; tc < ct; ++tc)
        CHECK(owner[((size_t)k * m + i) * ct + tc] >= 0, "3d n=%d: row %d plane %d tile %d uncovered\n", n, i, k, tc);
  if (fails) return;
  for (int idx = 0; idx < (int)s.size(); ++idx) {
    int nb[7];
    flow3_neighbours(idx, n, bands, ct, nb);
    const std::set<int> ok(nb, nb + 7);
    const Tile& t = s[idx];
    const int k = t.row0 / m, i0 = t.row0 - k * m, i1 = i0 + t.nrows, tc = (t.col0 - 1) / kWarpCols;
    auto need = [&](int kk, int ii, int cc) {
      if (kk < 1 || kk > n || ii < 1 || ii > n || cc < 0 || cc >= ct) return;  // shell or outside
      const int o = owner[((size_t)kk * m + ii) * ct + cc];
      CHECK(ok.count(o), "3d n=%d bands=%d: strip %d reaches strip %d, not a listed neighbour\n", n, bands, idx, o);
    };
    for (int i = i0; i < i1; ++i) {
      need(k, i - 1, tc);
      need(k, i + 1, tc);
      need(k - 1, i, tc);
      need(k + 1, i, tc);
      need(k, i, tc - 1);  // first packed column's west neighbour
      need(k, i, tc + 1);  // last packed column's east neighbour
    }
  }
}

static void check9(int n, int warps) {
  const Layout L = Layout::make(n);
  const int ct = L.col_tiles(), arows = (n + 1) >> 1, qrows = arows + 2;
  std::vector<Tile> s;
  const int bands = build_strips9(n, ct, warps, &s);
  CHECK((long)s.size() == (long)bands * ct, "9pt n=%d: %zu strips\n", n, s.size());
  std::vector<int> owner((size_t)qrows * ct, -1);
  for (int idx = 0; idx < (int)s.size(); ++idx) {
    const Tile& t = s[idx];
    const int a0 = t.row0, a1 = a0 + t.nrows, tc = (t.col0 - 1) / kWarpCols;
    CHECK(t.col0 == 1 + tc * kWarpCols && tc == idx % ct, "9pt n=%d strip %d: column tile\n", n, idx);
    CHECK(a0 >= 1 && a1 > a0 && a1 <= arows + 1, "9pt n=%d strip %d: rows\n", n, idx);
    CHECK(a0 - 1 >= 0 && a1 <= qrows - 1, "9pt n=%d strip %d: halo rows\n", n, idx);
    CHECK(t.col0 - 1 + kOff >= 0 && t.col0 + kWarpCols + kOff < L.pitch, "9pt n=%d strip %d: halo columns\n", n, idx);
    for (int a = a0; a < a1; ++a) {
      int& o = owner[(size_t)a * ct + tc];
      CHECK(o == -1, "9pt n=%d: quarter row %d tile %d in two strips\n", n, a, tc);
      o = idx;
    }
  }
  for (int a = 1; a <= arows; ++a)
    for (int tc = 0; tc < ct; ++tc) CHECK(owner[(size_t)a * ct + tc] >= 0, "9pt n=%d: row %d uncovered\n", n, a);
  if (fails) return;
  for (int idx = 0; idx < (int)s.size(); ++idx) {
    int nb[9];
    flow9_neighbours(idx, bands, ct, nb);
    const std::set<int> ok(nb, nb + 9);
    const Tile& t = s[idx];
    const int a0 = t.row0, a1 = a0 + t.nrows, tc = (t.col0 - 1) / kWarpCols;
    for (int a = a0; a < a1; ++a)
      for (int da = -1; da <= 1; ++da)      // quarter rows a - PI and a + 1 - PI, PI in {0, 1}
        for (int dc = -1; dc <= 1; ++dc) {  // columns b - PJ .. b + 1 - PJ reach the next tiles
          const int aa = a + da, cc = tc + dc;
          if (aa < 1 || aa > arows || cc < 0 || cc >= ct) continue;
          const int o = owner[(size_t)aa * ct + cc];
          CHECK(ok.count(o), "9pt n=%d bands=%d: strip %d reaches strip %d, not a listed neighbour\n", n, bands, idx, o);
        }
  }
}

int main() {
  const int warps[] = {1, 7, 100, 608, 1824, 5472};
  const int n3[] = {1, 2, 3, 5, 8, 9, 16, 17, 33, 64, 65, 130, 255, 256, 257, 259, 300, 515};
  const int n9[] = {1, 2, 3, 4, 7, 16, 37, 100, 129, 255, 256, 257, 300, 517, 1030, 4096};
  long cases = 0;
  for (int w : warps) {
    for (int n : n3) {
      check3(n, w);
      ++cases;
    }
    for (int n : n9) {
      check9(n, w);
      ++cases;
    }
  }
  std::printf("strips: %ld failures over %ld cases\n", fails, cases);
  return fails ? 1 : 0;
}
