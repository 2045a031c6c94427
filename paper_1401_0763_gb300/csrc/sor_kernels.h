// Host-side launch interface of the SOR kernels (sor_kernels.cu).
#pragma once
#include <cuda_runtime.h>

#include "sor_device.cuh"

namespace sorgb {

enum SweepKind : int { kSweepPlain64 = 0, kSweepPlain32 = 1, kSweepInner32 = 2 };
// dbuf argument of launch_resid: each slot's own SlotDesc::dbuf (slots whose
// inner sweep counts differ end their corrections in different buffers).
constexpr int kDbufPerSlot = -1;

// kResidRefine64 applies the pending correction (k_correct) before the
// residual; kResidRefine64Fixed omits it (the inner sweeps applied it).
enum ResidKind : int {
  kResidFinal64 = 0,
  kResidFinal32 = 1,
  kResidCheck64 = 2,
  kResidCheck32 = 3,
  kResidRefine64 = 4,
  kResidRefine64Fixed = 5
};

struct PackArgs {
  const double* u0;  // natural (n+2)^2, device
  const double* f;   // natural n^2 interior, device, or null
  int n, pitch;
  double h2;         // h*h, h = 1/(n+1)
  bool fp32;         // x / g arrays are FP32
  void* x[2][2];     // iterate buffers to fill (null entries skipped)
  void* g[2];        // sweep rhs h^2 f in the iterate's type (null: none)
  double* g64[2];    // h^2 f in FP64 (null: none)
  double* u[2][2];   // FP64 solution buffers to fill (refine; null entries skipped)
  SlotState* state;  // receives bmax_bits (must be zeroed before)
};

cudaError_t launch_pack(const PackArgs& a, cudaStream_t s);
cudaError_t launch_unpack(const void* c0, const void* c1, bool fp32, int n, int pitch, double* out, cudaStream_t s);
cudaError_t launch_sweep(SweepKind kind, const SlotDesc* slots, SlotState* states, const Tile* tiles, int ntiles,
                         int grid, int colour, int sweep, cudaStream_t s);
// Constants of one FP64 colour phase of the rescaled formulation:
//   X' = alpha * X + beta * (pair-sum of neighbours) + gamma * g,
// with |change| measured as |X' - dscale * X| (last iteration of a chunk only);
// the phase rewrites its colour's Dirichlet ring cells at nscale x value.
struct FastPhaseArgs {
  double alpha, beta, gamma, dscale;
  double nscale;  // scale at which the next phase reads this phase's colour (its ring cells are written so)
  int last;
};
// Saves the unscaled Dirichlet ring cells of slot 0's colour arrays into
// slots[0].ring (needed by the FP64 default phases, which rewrite the ring at
// the scale of the next phase).
cudaError_t launch_ring_save(const SlotDesc* slots, cudaStream_t s);
// Kernel launches issued by the calling thread through these wrappers.
unsigned long long kernel_launch_count();
void count_kernel_launches(int k);
// Resident blocks per SM of the FP64 phase kernel (sizes its persistent grid).
int fast_blocks_per_sm();
// The 2L FP64 phases of a chunk in one cooperative launch: one warp per strip
// of a table of rows x ct strips (row-major), neighbour-to-neighbour progress
// counters (nstrips unsigned, zeroed before the launch) instead of a grid
// barrier; `phases` holds nphases packed phase records (fast_phase_pack).
int fast_chain_blocks_per_sm();
cudaError_t launch_fast_chain(const SlotDesc* slots, SlotState* states, const Tile* strips, int nstrips, int ct,
                              const void* phases, int nphases, unsigned* progress, bool has_g, int grid,
                              cudaStream_t s);
size_t fast_phase_bytes();
void fast_phase_pack(const FastPhaseArgs& a, void* out);
// ntiles counts warp strips (one warp each); grid <= 0: one warp per strip.
cudaError_t launch_sweep_fast64(const SlotDesc* slots, SlotState* states, const Tile* tiles, int ntiles, int grid,
                                int colour, const FastPhaseArgs& a, bool has_g, cudaStream_t s);
// FP32 phases fused over nt <= T iterations per launch (temporal blocking).
// Two kernel families compute the same iterations bit for bit:
//   kFusedTile (sor_tile.cu): T iterations per shared-memory tile pass, tiles
//     of tile_out_rows() output rows; depths 2, 3, 4, 6, 8;
//   kFusedWave (sor_wf.cu): a register wavefront per warp streaming down a
//     segment of rows (wave_seg_rows by default); depths 2 .. 5.
// Tiles are out_rows x fused_out_cols(kind, T) output packed columns starting
// at column 1.  inner: correction sweeps of defect correction (src = buffer
// holding d, sweep0 = index of the first sweep of this launch within the
// correction); otherwise plain FP32 iterations (buffer and iteration count
// from the slot state).  Writes buffer src ^ 1.
enum FusedKind : int { kFusedTile = 0, kFusedWave = 1 };
bool fused_depth_supported(int kind, int T);
int fused_out_cols(int kind, int T);
// Output rows per tile: the tile family's fixed height; for the wavefront
// `seg` when positive, else its default for an n x n plate on sm_count SMs.
int fused_out_rows(int kind, int n, int T, int sm_count, int seg);
// Opts the kernels of depth T into their shared memory (call outside graph capture).
cudaError_t fused_prepare(int kind, int T);
// correct (inner sweeps, families with fused_corrects(kind)): the launch that
// ends a slot's inner sweeps adds the final correction to u itself.
cudaError_t launch_fused(int kind, bool inner, int T, const SlotDesc* slots, SlotState* states, const Tile* tiles,
                         int ntiles, int grid, int nt, int src, int sweep0, cudaStream_t s, bool correct = false);
bool fused_corrects(int kind);
// the two families
bool tile_depth_supported(int T);
int tile_out_cols(int T);
int tile_out_rows();
cudaError_t tile_prepare(int T);
cudaError_t launch_sweep_tile(bool inner, int T, const SlotDesc* slots, SlotState* states, const Tile* tiles,
                              int ntiles, int grid, int nt, int src, int sweep0, cudaStream_t s, bool correct);
bool wave_depth_supported(int T);
int wave_out_cols(int T);
int wave_warps_per_sm(int T);
int wave_seg_rows(int n, int T, int sm_count);
cudaError_t wave_prepare(int T);
cudaError_t launch_sweep_wave(bool inner, int T, const SlotDesc* slots, SlotState* states, const Tile* tiles,
                              int ntiles, int grid, int nt, int src, int sweep0, cudaStream_t s);
// Whole plain solve of a small grid inside one thread-block cluster (one
// launch runs every iteration and the stopping test); exact-order update.
bool cluster_solve_fits(bool fp32, int n, int pitch);
cudaError_t launch_cluster_solve(bool fp32, int n, int pitch, const SlotDesc* slots, SlotState* states, int slot,
                                 cudaStream_t s);
// Largest plates solved in one launch (grid or cluster) by default.
constexpr int kGridMaxN64 = 384;
constexpr int kGridMaxN32 = 768;
// Whole plain solve of a small plate on a cooperative grid of many SMs, one
// band of rows per block (sor_grid.cu); exact-order update, max|change| stop
// only.  `sync` is grid_sync_bytes() of device memory (zeroed by the launch).
bool grid_solve_fits(bool fp32, int n, int pitch, int sm_count);
size_t grid_sync_bytes();
cudaError_t launch_grid_solve(bool fp32, int n, int pitch, int sm_count, const SlotDesc* slots, SlotState* states,
                              int slot, void* sync, cudaStream_t s);
// The same solves without grid barriers: tagged edge-row exchanges between
// neighbouring bands and a stop test that an extra block decides behind the
// sweeps (sor_grid.cu).  `sync` holds grid_flow_sync_bytes() (zeroed by the
// launch); 0 bytes or a false fit: the plate does not fit this form.
bool grid_flow_fits(bool fp32, int n, int pitch, int sm_count);
size_t grid_flow_sync_bytes(bool fp32, int n, int pitch, int sm_count);
cudaError_t launch_grid_flow(bool fp32, int n, int pitch, int sm_count, const SlotDesc* slots, SlotState* states,
                             int slot, void* sync, size_t sync_bytes, cudaStream_t s);
cudaError_t launch_resid(ResidKind kind, const SlotDesc* slots, SlotState* states, const Tile* tiles, int ntiles,
                         int grid, int dbuf, cudaStream_t s);

}  // namespace sorgb
