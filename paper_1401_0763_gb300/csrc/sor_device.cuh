// Device-side data structures and the colour-split storage layout.
//
// Storage ("shifted checkerboard packing").  Cell (i, j) of the (N+2)^2 grid
// has colour c = (i + j) & 1 (red = 0 when i+j is even, black = 1; paper
// Section 3.1, Figure 1) and is stored in colour array c at row i, packed
// column q = (j + 1) >> 1, element  i * pitch + q + kOff.  With
// s = (i + c) & 1 (equivalently s = j & 1) the natural column is j = 2q - s,
// and the four neighbours of (i, q) live in the other colour array o at
//     N = o[i-1][q],  S = o[i+1][q],  W = o[i][q - s],  E = o[i][q - s + 1].
// Interior cells are exactly 1 <= i <= N and 1 <= q <= (N + s) / 2, so every
// row of either colour starts its interior at q = 1, which kOff places on a
// 16-byte boundary: rows stream as aligned float4 / double2 vectors and the
// red and black phases (Section 3.1) become branch-free, unit-stride sweeps
// (the loop restructuring of Figure 2 carried to the data layout).
#pragma once
#include <cstddef>
#include <cstdint>

namespace sorgb {

constexpr int kOff = 3;                // element offset of packed column 0
constexpr int kVec = 4;                // consecutive packed columns per thread
constexpr int kWarpCols = 32 * kVec;   // 128 packed columns per warp / tile
constexpr int kWarpsY = 4;             // warps per block, stacked in rows
constexpr int kThreads = 32 * kWarpsY; // 128 threads per block
constexpr int kTileRows = 32;          // rows per sweep tile (8 per warp)

struct Layout {
  int n;      // interior side
  int rows;   // n + 2
  int qmax;   // floor((n + 1) / 2): largest interior packed column over both parities
  int qw;     // qmax + 2: packed columns 0 .. qmax + 1 (ring included)
  int pitch;  // elements per row (multiple of 32)

  static Layout make(int n) {
    Layout L;
    L.n = n;
    L.rows = n + 2;
    L.qmax = (n + 1) / 2;
    L.qw = L.qmax + 2;
    int tiles = (L.qmax + kWarpCols - 1) / kWarpCols;
    int need = kOff + tiles * kWarpCols + 2 * kVec;  // whole tiles plus one vector of halo stay in the row
    L.pitch = (need + 31) / 32 * 32;
    return L;
  }
  size_t elems() const { return (size_t)rows * (size_t)pitch; }
  int col_tiles() const { return (qmax + kWarpCols - 1) / kWarpCols; }
  int row_tiles() const { return (n + kTileRows - 1) / kTileRows; }
};

// Kinds of work a slot carries.
enum SlotKind : int { kPlain64 = 0, kPlain32 = 1, kRefine = 2 };
enum StopKind : int { kStopDelta = 0, kStopResid = 1 };

// One solve ("slot") as seen by the kernels.  Immutable while the slot is
// active.  All arrays use the layout above with this slot's n / pitch.
struct SlotDesc {
  void* x[2][2];        // iterate [buffer][colour]: plain -> u in FP64 / FP32; refine -> correction d (FP32)
  void* g[2];           // [colour] right side used by the sweeps: plain -> h^2 f (same type as x) or null;
                        //          refine -> scaled residual r~ rounded to FP32
  double* u[2][2];      // refine: FP64 solution [buffer][colour]
  const double* g64[2]; // h^2 f in FP64 [colour] or null (residual passes)
  const double* ring[2]; // FP64 default path: unscaled Dirichlet ring cells of each colour array, saved
                         // after packing: [row 0: pitch][row N+1: pitch][column q = 0: N+2 rows]
                         // [east ring column: N+2 rows]; null elsewhere
  int n, pitch, qmax, kind;
  int sweep_tiles;      // tiles of this slot in one sweep launch
  int resid_tiles;      // tiles of this slot in one residual launch
  int K, max_iters, stop, inner;
  int stall;            // residual tests without a new minimum that end the solve (0 = never)
  int dbuf;             // refine: buffer of x holding the correction after a step's inner sweeps
                        // (read by launches given kDbufPerSlot)
  float a32, b32;       // (float)(1 - w), (float)(w / 4)
  double a64, b64;      // 1 - w, w / 4
  double tol;
};

// Mutable per-slot state, device resident.
struct SlotState {
  unsigned long long dmax_bits;  // max |change| of the current iteration (bits of a non-negative double)
  unsigned long long rmax_bits;  // max |r~| of the current residual pass
  unsigned long long bmax_bits;  // max |b~| (right side with the boundary moved in), set at pack time
  unsigned int arrive;           // tile arrivals of the current sweep launch
  unsigned int arrive_res;       // tile arrivals of the current residual launch
  int iters;                     // red-black iterations completed
  int outer;                     // corrections applied (refine)
  int done;                      // 1: no further work (converged, capped or failed)
  int converged;
  int xbuf;                      // buffer of x holding the current iterate
  int ubuf;                      // buffer of u holding the current solution (refine)
  int checked_iter;              // iteration of the last residual test
  int error;                     // nonzero: device-side consistency failure
  int stall_run;                 // residual tests in a row without a new minimum, within 4x of it
  int reserved_;
  double best_rho;               // smallest rho so far (+inf before the first test)
  double last_dmax;              // m_k of the last iteration that measured it (-1 if none)
  double last_rho;               // relative residual of the last residual pass (-1 if none)
  unsigned long long umax_bits;  // max |u0| over the whole array (ring and interior), set at pack time
  unsigned long long gmax_bits;  // max |h^2 f| over the interior, set at pack time
};

// SlotState::error values: 1 = a consistency check of the kernels failed;
// kErrBounds = a device-side index check of the debug build refused an access.
constexpr int kErrBounds = 2;

// A tile of work: slot index, first row, first packed column, row count.
struct Tile {
  int slot, row0, col0, nrows;
};

// Residual-pass roles.
enum ResidRole : int {
  kResidFinal = 0,   // measure rho of the current iterate (no decisions)
  kResidCheck = 1,   // plain residual stop: test rho < tol when iters % K == 0
  kResidRefine = 2   // refine: apply the pending correction, write r~, test rho < tol
};

}  // namespace sorgb
