// Warp strips of the data-flow kernels (cube and four-colour 9-point) and
// the neighbour sets their work items wait for.  Host code builds the strip
// tables; the kernels derive a strip's neighbours from its number with the
// same functions, which a host harness checks against brute force (every
// cell a strip's stencil reads, or whose reader it could overwrite, lies in
// the strip itself or in one of the listed neighbours).
#pragma once
#include <algorithm>
#include <vector>

#include "sor_device.cuh"

#ifdef __CUDACC__
#define SOR_HD __host__ __device__ __forceinline__
#else
#define SOR_HD inline
#endif

namespace sorgb {

// Cube strips: every plane k = 1..N cut into `bands` row bands of about 32
// rows (at least 8, and at least one strip per resident warp), times the
// 128-column tiles.  Strip number ((k - 1) * bands + band) * ct + tile;
// row0 = k (N+2) + first row.  Returns `bands`.
inline int build_strips3(const Layout& L, int warps, std::vector<Tile>* out) {
  const int n = L.n, m = n + 2, ct = L.col_tiles();
  const long long per_band = (long long)n * ct;
  int b = std::max(n / 32, (int)((warps + per_band - 1) / per_band));
  b = std::max(1, std::min(b, std::max(1, n / 8)));
  for (int k = 1; k <= n; ++k)
    for (int r = 0; r < b; ++r) {
      const int a0 = 1 + (int)((long long)r * n / b), a1 = 1 + (int)((long long)(r + 1) * n / b);
      for (int t = 0; t < ct; ++t) out->push_back(Tile{0, k * m + a0, 1 + t * kWarpCols, a1 - a0});
    }
  return b;
}

// The strips a cube strip t waits for: itself and its face neighbours (the
// planes below and above, the row bands above and below, the column tiles
// left and right; -1 = none).  The 7-point stencil reaches no others.
SOR_HD void flow3_neighbours(int t, int n, int bands, int ct, int (&nb)[7]) {
  const int per_plane = bands * ct;
  const int kp = t / per_plane, r = t - kp * per_plane, band = r / ct, tc = r - band * ct;
  nb[0] = t;
  nb[1] = kp > 0 ? t - per_plane : -1;
  nb[2] = kp + 1 < n ? t + per_plane : -1;
  nb[3] = band > 0 ? t - ct : -1;
  nb[4] = band + 1 < bands ? t + ct : -1;
  nb[5] = tc > 0 ? t - 1 : -1;
  nb[6] = tc + 1 < ct ? t + 1 : -1;
}

// 9-point strips: quarter rows 1 .. (N+1)/2 cut into bands of about 32 rows
// (at least 8, at least one strip per resident warp), times the 128-column
// tiles.  Strip number band * ct + tile.  Returns `bands`.
inline int build_strips9(int n, int ct, int warps, std::vector<Tile>* out) {
  const int arows = (n + 1) >> 1;
  int b = std::max(arows / 32, (warps + ct - 1) / ct);
  b = std::max(1, std::min(b, std::max(1, arows / 8)));
  for (int r = 0; r < b; ++r) {
    const int a0 = 1 + (int)((long long)r * arows / b), a1 = 1 + (int)((long long)(r + 1) * arows / b);
    for (int t = 0; t < ct; ++t) out->push_back(Tile{0, a0, 1 + t * kWarpCols, a1 - a0});
  }
  return b;
}

// The strips a 9-point strip t waits for: itself and the eight around it
// (the diagonal couplings reach the corner strips; -1 = none).
SOR_HD void flow9_neighbours(int t, int bands, int ct, int (&nb)[9]) {
  const int band = t / ct, tc = t - band * ct;
  const bool up = band > 0, down = band + 1 < bands, left = tc > 0, right = tc + 1 < ct;
  nb[0] = t;
  nb[1] = up ? t - ct : -1;
  nb[2] = down ? t + ct : -1;
  nb[3] = left ? t - 1 : -1;
  nb[4] = right ? t + 1 : -1;
  nb[5] = up && left ? t - ct - 1 : -1;
  nb[6] = up && right ? t - ct + 1 : -1;
  nb[7] = down && left ? t + ct - 1 : -1;
  nb[8] = down && right ? t + ct + 1 : -1;
}

}  // namespace sorgb

#undef SOR_HD
