// Shared-memory tile kernels for the large axis levels of the FP32 inner cycle
// (tiles.cu): a block stages a tile of the level plus a halo in shared memory with one
// TMA load per array and runs several relaxation phases on it, so that data move
// between HBM and the SMs once per fused group of steps instead of once per step.
//
//   presmooth: nu1 (1 or 2) red-black sweeps from u = 0, f -> u   (reads f, writes u)
//   sweep:     one red-black sweep, u -> uout                       (reads u, f, writes uout)
//   residual + restriction (red-black, axis -> rotated):          (reads u, f, writes f_coarse)
//
// Every node's arithmetic is that of the per-step kernels (same terms, same order,
// same rounding), so the fused kernels give the same bits.
#pragma once

#include <cuda.h>

#include "kernels.h"

namespace nsmg {

// Tensor maps and geometry of one eligible level (built once per handle at set-up).
struct TileLevel {
  bool on = false;
  int reach = 0;        // stencil reach (1: 5-point cross, 2: 9-point fourth-order cross)
  int nt = 0;           // 5 or 9
  int nu1 = 0;          // presmooth sweeps (1 or 2); 0: no fused presmooth
  bool rot = false;     // a rotated level (brick storage, colours by rows)
  dim3 grid;            // tiles
  CUtensorMap f_pre;    // f with the presmooth halo
  CUtensorMap u_sw, t_sw, f_sw;  // u, t and f with the one-sweep halo
  CUtensorMap u_rr, f_rr;        // u and f with the residual + restriction halo
};

// Whether level L (FP32) can use the tile kernels: a level of at least kTileMinRows rows
// with Dirichlet boundaries and no bfloat16 rounding whose interior stencil is a 5-point
// or 9-point cross (axis levels) or the first Galerkin 9-point stencil (rotated levels).
bool tile_eligible(const LevelPair<float>& L);
// Build the tensor maps of level L over its arrays u, t, f. false if the CUDA driver's
// tensor-map encoder is unavailable or rejects a map.
bool tile_setup(TileLevel& T, const LevelPair<float>& L, float* u, float* t, float* f, int nu1);

// u = nu1 red-black sweeps from zero on f (u's boundary entries are written as 0).
cudaError_t launch_tile_presmooth(const TileLevel& T, const LevelPair<float>& L, bool exact, float* u, int* status,
                                  cudaStream_t s);
// One red-black sweep: src is u (from_t = false) or t (from_t = true); the result goes
// to the other array.
cudaError_t launch_tile_sweep(const TileLevel& T, const LevelPair<float>& L, bool exact, bool from_t, float* uout,
                              int* status, cudaStream_t s);
// f_coarse = R (f - L u) for red-black coarsening (axis level -> its black points, or
// rotated level -> its axis level); with tc also the coarse level's first half-sweep
// from zero (as launch_restrict).
cudaError_t launch_tile_res_restrict(const TileLevel& T, const LevelPair<float>& L, const LevelPair<float>& Lc,
                                     bool exact, float* fc, float* tc, int* status, cudaStream_t s);

// Bit set in the handle's status word when a bounded wait in a tile kernel gave up.
constexpr int kStatusTmaTimeout = 1;

}  // namespace nsmg
