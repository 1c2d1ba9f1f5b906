// Launch wrappers for the multigrid kernels (kernels.cu). Every wrapper enqueues
// on `s` and returns the launch status.
#pragma once

#include "levels.h"

namespace nsmg {

// Host copy + device copy of a level description.
template <typename T>
struct LevelPair {
  LevelDev<T> h;            // host copy (launch geometry, scalars)
  LevelDev<T>* d = nullptr;  // device copy (read by kernels)
};

template <typename T>
cudaError_t launch_half_sweep(const LevelPair<T>& L, bool exact, const T* uin, const T* f, T* uout,
                              int red, cudaStream_t s);
template <typename T>
cudaError_t launch_jacobi(const LevelPair<T>& L, bool exact, const T* uin, const T* f, T* uout,
                          cudaStream_t s);
template <typename T>
cudaError_t launch_apply(const LevelPair<T>& L, bool exact, const T* u, T* out, cudaStream_t s);
template <typename T>
cudaError_t launch_residual(const LevelPair<T>& L, bool exact, const T* u, const T* f, T* d,
                            cudaStream_t s);
// With tc: also the coarse level's first half-sweep from u = 0 (as launch_first_half_zero).
template <typename T>
cudaError_t launch_restrict(const LevelPair<T>& Lf, const LevelPair<T>& Lc, int transfer, bool exact,
                            const T* d, T* fc, cudaStream_t s, T* tc = nullptr);
// uf = uin + P vc (uin = nullptr: in place, uf += P vc).
template <typename T>
cudaError_t launch_prolong_add(const LevelPair<T>& Lf, const LevelPair<T>& Lc, int transfer,
                               bool exact, T* uf, const T* vc, cudaStream_t s, const T* uin = nullptr);
// One full red-black sweep uin -> uout in a single kernel (shared-memory tiles).
template <typename T>
cudaError_t launch_sweep_fused(const LevelPair<T>& L, bool exact, const T* uin, const T* f, T* uout,
                               cudaStream_t s);
template <typename T>
cudaError_t launch_coarsest(int64_t idx, T a, int zero_mean, const T* f, T* u, cudaStream_t s);

// Exact coarsest solve with m > 1 unknowns (Dirichlet): x = G^T (G d), G = L^-1 the
// inverse Cholesky factor of the coarsest operator, formed on the host at set-up in a
// fixed order. y_i = G_i0 d_0 + ... + G_ii d_i, then x_i = G_ii y_i + ... + G_m-1,i y_m-1,
// each sum from its first product with k ascending (separately rounded when exact).
template <typename T>
struct DenseCoarse {
  const T* ga;     // ga[k * m + i] = G_ik (k <= i): reads coalesced over i
  const T* gb;     // gb[k * m + i] = G_ki (k >= i)
  const int2* ij;  // lattice coordinates (i, j) of unknown k, row-major (j, then i)
  int32_t m;       // unknowns; 0: one unknown, solved by the division
};
// Dense coarsest solve on level L's storage: u = G^T (G f), y (the level's d array)
// holds G f in between. One block.
template <typename T>
cudaError_t launch_coarsest_dense(const DenseCoarse<T>& C, const LevelPair<T>& L, bool exact, const T* f, T* y, T* u,
                                  cudaStream_t s);

// Sum of squares of d = f - L u over interior nodes of an axis level, in FP64:
// per-block partial sums into `partial` (size >= resnorm_blocks(L)), then one
// block adds the partials in a fixed order into *out. Deterministic.
template <typename T>
int resnorm_blocks(const LevelPair<T>& L);
template <typename T>
cudaError_t launch_resnorm(const LevelPair<T>& L, bool exact, const T* u, const T* f,
                           double* partial, double* out, cudaStream_t s);
// Sum of squares of f over interior nodes (same reduction order).
// t = the first half-sweep (colour red) from u = 0: red unknowns 0 + f omega / a_pp, others 0.
template <typename T>
cudaError_t launch_first_half_zero(const LevelPair<T>& L, const T* f, T* t, int red, cudaStream_t s);
// out = ||f - L u||^2 (as launch_resnorm) and, from the same residual, uout = u with the
// nodes of colour `red` relaxed: the first half-sweep of a following cycle.
template <typename T>
cudaError_t launch_resnorm_red(const LevelPair<T>& L, bool exact, const T* u, const T* f, T* uout, int red,
                               double* partial, double* out, cudaStream_t s);
template <typename T>
cudaError_t launch_sumsq(const LevelPair<T>& L, const T* f, double* partial, double* out,
                         cudaStream_t s);

// Zero the boundary entries of an axis-level array.
template <typename T>
cudaError_t launch_zero_boundary(const LevelPair<T>& L, T* u, cudaStream_t s);
// Copy the boundary ring of src (a level's storage) into dst.
template <typename T>
cudaError_t launch_copy_boundary(const LevelPair<T>& L, const T* src, T* dst, cudaStream_t s);

// Refinement step, finest level (FP64 grid L, FP32 grid L32 of the same nodes with its
// own row pitch): r32 = fl32((f - L u) * scale), *out = sum of (f - L u)^2 (two launches).
// With t32: also the first half-sweep (red) of the FP32 cycle from e = 0 into t32.
cudaError_t launch_ir_residual(const LevelPair<double>& L, bool exact, const double* u, const double* f,
                               const LevelPair<float>& L32, float* r32, double scale, double* partial,
                               double* out, cudaStream_t s, int bf16 = 0, float* t32 = nullptr);
// u += e * inv_scale on interior nodes (e in the FP32 finest level's storage).
cudaError_t launch_ir_update(const LevelPair<double>& L, const LevelPair<float>& L32, double* u, const float* e,
                             double inv_scale, cudaStream_t s);

// ---- small-level tail: one thread block runs a whole sub-cycle ---------------
constexpr int kTailMaxLevels = 40;
// kOpSmooth with z = 1: the first red-black sweep from u = 0 (the level's u is not zeroed
// first; its red half-sweep needs no stencil).
enum TailOp : int32_t { kOpZero = 0, kOpSmooth = 1, kOpResRestrict = 2, kOpCoarsest = 3, kOpProlong = 4 };

// Levels and buffers the tail program refers to (device-resident).
template <typename T>
struct TailDesc {
  const LevelDev<T>* L[kTailMaxLevels];
  T* u[kTailMaxLevels];
  T* t[kTailMaxLevels];
  T* f[kTailMaxLevels];
  T* d[kTailMaxLevels];
  int32_t transfer[kTailMaxLevels];
  int32_t smoother;  // mg_smoother
  int64_t coarsest_idx;
  T coarsest_a;
  int32_t coarsest_zero;  // periodic single node: the zero-mean solution 0
  DenseCoarse<T> dense;   // m > 0: the coarsest level's dense solve
  // shared-memory-resident variant: per level, element offsets of u, t, f, d in the
  // block's shared memory (compact rows x cols layout) and the number of levels held
  int32_t sm_u[kTailMaxLevels], sm_t[kTailMaxLevels], sm_f[kTailMaxLevels], sm_d[kTailMaxLevels];
  int32_t sm_top;     // first level held (the sub-cycle's top level)
  int32_t sm_elems;   // shared-memory elements of the level arrays
  int32_t nlev;       // levels of the hierarchy (those from sm_top on are held)
};

// The same op list, with every level from sm_top down held in one block's shared
// memory (u and f of the top level are loaded at start, u written back at the end).
template <typename T>
cudaError_t launch_tail_smem(const TailDesc<T>* desc, int sm_elems, int nst, const int4* prog, int nops, bool exact,
                             cudaStream_t s);
// Dynamic shared memory of the shared-memory tail: the level arrays (sm_elems values)
// and the interior stencils of its nst levels; at most kTailSmemMaxBytes.
template <typename T>
size_t tail_smem_bytes(int sm_elems, int nst);
constexpr size_t kTailSmemMaxBytes = 227 * 1024;

// Run `nops` ops (x = TailOp, y = level) in order inside one thread-block cluster of
// `ctas` CTAs, with a cluster barrier after each phase. Op semantics match the
// per-level kernels bit for bit.
template <typename T>
cudaError_t launch_tail(int ctas, const TailDesc<T>* desc, const int4* prog, int nops, bool exact, cudaStream_t s);
// Largest tail cluster the current device can schedule (16, 8, 4, 2 or 1 CTAs).
template <typename T>
int tail_ctas(bool exact);

// ---- batched level-synchronous schedule ----------------------------------------
// One problem's level l as seen by a batched step kernel.
template <typename T>
struct BatchLevel {
  const LevelDev<T>* L;   // level l
  const LevelDev<T>* Lc;  // level l + 1 (null at the coarsest)
  T* u;                   // level-l arrays (level 0: refinement correction / caller's u)
  T* t;
  T* f;
  T* d;
  T* uc;                  // level l + 1 arrays
  T* fc;
  int32_t transfer;
  int32_t problem;        // index into the batch's per-problem arrays
  int32_t cols, rows, n, kind;
  int32_t tiles_x, ctiles_x;  // tiles per row of tiles on level l / level l + 1
  int64_t coarsest_idx;   // of level l + 1 when it is the problem's coarsest level
  T coarsest_a;
  DenseCoarse<T> dense;   //   m > 0: its dense solve (y in dc)
  T* dc;                  // level l + 1's d array
  float* r32;             // finest level, mixed precision: FP32 residual (inner right-hand side)
  float* e32;             //   and FP32 correction
  int32_t pitch32;        //   row pitch of those FP32 arrays (padded to 32 elements)
};

enum BatchOp : int32_t {
  kBZero = 0, kBHalfRed = 1, kBHalfBlack = 2, kBResidual = 3, kBRestrict = 4, kBProlong = 5, kBCoarsest = 6,
  kBHalfRedZero = 7,  // kBHalfRed from u = 0 (no stencil; replaces kBZero + kBHalfRed, same bits)
  kBCoarsestDense = 8  // kBCoarsest for coarsest levels with several unknowns (one block per problem)
};

// A tile is 64 storage columns (2 per thread, so a thread holds one red and one black
// node of an axis row) by 8 x rpt rows; a block of 32 x 8 threads handles one tile of
// one problem. Block b belongs to the entry e with prefix[e] <= b < prefix[e + 1].
constexpr int kBatchCols = 64;
inline int batch_tiles(int cols, int rows, int rpt) {
  return ((cols + kBatchCols - 1) / kBatchCols) * ((rows + 8 * rpt - 1) / (8 * rpt));
}

// One step (BatchOp) for every problem of a level list (`entries`, count ne, device
// memory); `prefix` (ne + 1 ints) is the exclusive prefix sum of the tiles each entry
// needs (level l's storage, or level l + 1's for kBRestrict). Problems with
// active[problem] == 0 skip. kBCoarsest runs one thread per entry instead.
template <typename T>
cudaError_t launch_batch_step(int op, const BatchLevel<T>* entries, const int* prefix, int ne, int total_tiles,
                              int rpt, const int* active, bool exact, cudaStream_t s);
// Finest levels of a batch (FP64 entries, rpt = 1 tiles). mode 0: r = f - L u,
// r32 = fl32(r * scale[problem]) and partial[tile] = sum of r^2; mode 1: partial =
// sum of f^2; mode 2: partial = sum of r^2 only. Then norm2[problem] = the entry's partials added in a fixed order.
cudaError_t launch_batch_norms(int mode, const BatchLevel<double>* entries, const int* prefix, int ne,
                               int total_tiles, const int* active, const double* scale, bool exact,
                               double* partial, double* norm2, cudaStream_t s);
// u += e32 / scale[problem] on the finest levels.
cudaError_t launch_batch_ir_update(const BatchLevel<double>* entries, const int* prefix, int ne, int total_tiles,
                                   const int* active, const double* scale, cudaStream_t s);

}  // namespace nsmg
