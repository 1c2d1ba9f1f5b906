/*
 * nsmg.h — C ABI of the GB300 multigrid library for 2D Poisson problems with
 * nonstandard (red-black, "rotated-grid") or standard coarsening.
 *
 * Method: Liu & Henshaw, "Multigrid with nonstandard coarsening",
 * arXiv:2008.03885. The problem statement is Sec. 2.1 (L_h u_h = f_h); the
 * fine operators are Eq. (L_h_2) and Eq. (L_h_2d_4o) (Sec. 2.3); coarse grids
 * are standard coarsening H = 2h (Eq. G_H_d) or red-black coarsening H = sqrt(2) h
 * (Sec. 4.3, Eq. G_r2), recursively (Sec. 4.4); transfers are Eq. (transfer_2d)
 * and Eq. (transfer_r2); coarse operators are the non-Galerkin / Galerkin /
 * G1 / Gn / G^(2) family of Sec. 2.3 and Sec. 4.4 (Eq. L_G_l); the smoother is
 * red-black relaxation, Eq. (S_rb), or weighted Jacobi (Sec. 5.3); the cycle is
 * the gamma-cycle of Sec. 2.2 (Algorithm "MG").
 *
 * Conventions shared by every call
 * --------------------------------
 * - Domain: the square [0, length]^2 (default the unit square), N cells per side (N a
 *   power of two, 4 <= N <= 16384), h = length/N, Eq. (G_h_N), with homogeneous Dirichlet boundary values (default) or
 *   periodic boundaries (mg_options.boundary), the setting of the paper's computed
 *   results (Sec. 2.2).
 * - Grid arrays on the finest level are caller-owned DEVICE pointers to
 *   (N+1) x (N+1) contiguous doubles, row-major with x fastest:
 *   a[j*(N+1) + i] is the node (i h, j h).
 *   Dirichlet: the unknowns are the interior nodes 0 < i, j < N; boundary entries
 *   of f are ignored and those of u are set to zero by mg_cycle / mg_solve, unless
 *   mg_options.dirichlet_data = 1 (second order), where they hold the data g and are
 *   kept.
 *   Periodic: the unknowns are the nodes 0 <= i, j < N (node N is node 0); row N
 *   and column N of u and f are neither read nor written. The periodic operator
 *   annihilates constants, so f must have zero mean over the unknowns (else the
 *   residual cannot drop below that mean's share of ||f||), and u is determined up
 *   to a constant: the coarsest level's exact solve is the zero-mean one, but
 *   relaxation moves the mean of the iterate, so compare solutions after removing
 *   their means.
 * - u is the initial guess and is overwritten with the new iterate.
 * - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *   Work is enqueued on it; calls with *_out arguments synchronise the stream
 *   before returning so that the outputs are valid.
 * - The handle owns every hierarchy buffer (allocated with cudaMalloc at setup,
 *   freed by mg_destroy). A handle is not thread-safe; different handles are
 *   independent.
 * - Errors are returned as mg_status, never by aborting. After an error other
 *   than MG_ERR_CUDA the handle stays usable; the content of u is unspecified.
 * - Relative residual = ||f - L_h u||_2 / ||f||_2 over interior nodes (the h^d
 *   weight of the paper's grid norm, Sec. 2.1, cancels).
 * - Floating-point evaluation order (precision MG_PREC_FP64, fma_contract = 0):
 *   every operator row (a_pq fixed) is split into groups of nonzeros of equal value;
 *   the groups are ordered by the row-major position of their first column and each
 *   group's columns in increasing row-major position; the row's value is
 *   sum_g a_g * (x_g1 + x_g2 + ...), every sum left to right and every product and
 *   sum rounded separately. Grid transfers sum their products in increasing position
 *   of the column. Relaxation is u + r * fl(omega / a_pp) with r = f - (A u). Two
 *   implementations that follow this order produce the same iterates bit for bit.
 */
#ifndef NSMG_H
#define NSMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MG_OK = 0,
  MG_ERR_INVALID = 1,       /* bad argument: size, enum, NULL pointer, level index */
  MG_ERR_UNSUPPORTED = 2,   /* valid request the library does not implement */
  MG_ERR_OOM = 3,           /* device allocation failed */
  MG_ERR_BUDGET = 4,        /* request exceeds a caller-set memory budget */
  MG_ERR_CUDA = 5,          /* a CUDA runtime call failed; the handle must be destroyed */
  MG_ERR_NONFINITE = 6,     /* a residual norm is NaN or Inf */
  MG_ERR_NOT_CONVERGED = 7, /* mg_solve reached max_cycles above rtol */
  MG_ERR_TIMEOUT = 8        /* a bounded device-side wait gave up */
} mg_status;

typedef enum {
  MG_COARSEN_STANDARD = 0, /* H = 2h, Eq. (G_H_d) */
  MG_COARSEN_REDBLACK = 1, /* H = sqrt(2) h, black points of the finer level, Eq. (G_r2) */
  MG_COARSEN_VARIABLE = 2  /* red-black for coarse levels 1 and 2, standard below (Sec. 4.4 "VC") */
} mg_coarsening;

typedef enum {
  MG_OP_NONGALERKIN = 0,        /* 5-point stencil with spacing H on every coarse level
                                   (for order 4 this is nG^(2), Eq. L_H_2d) */
  MG_OP_GALERKIN = 1,           /* L_{l+1} = R L_l P, Eq. (L_G_l); for order 4 the
                                   recursion starts from L_h^(2) (G^(2), Eq. L_H_2G_2d) */
  MG_OP_GALERKIN_G1 = 2,        /* Eq. (L_G1) stencil on every coarse level (Sec. 4.4 "G1") */
  MG_OP_GALERKIN_GN = 3,        /* Galerkin on level 1, non-Galerkin below (Sec. 4.4 "Gn") */
  MG_OP_GALERKIN_TRUE_HIGH = 4, /* Galerkin recursion from the order-4 (or 6) operator itself */
  MG_OP_NONGALERKIN_HIGH = 5    /* the fine operator's own stencil with spacing H on every coarse
                                   level: nG^(4) (Eq. L_H_4n_2d) for order 4, nG^(6) for order 6;
                                   the same as MG_OP_NONGALERKIN for order 2 */
} mg_coarse_op;

typedef enum {
  MG_SMOOTH_REDBLACK = 0, /* S = S^B S^R, Eq. (S_rb); Jacobi within a colour */
  MG_SMOOTH_JACOBI = 1    /* weighted Jacobi, Sec. 5.3 */
} mg_smoother;

typedef enum {
  MG_PREC_FP64 = 0,       /* every level in FP64 */
  MG_PREC_MIXED_FP32 = 1  /* FP64 residual/update, FP32 inner cycles (iterative refinement) */
} mg_precision;

typedef enum {
  MG_BOUNDARY_DIRICHLET = 0, /* u = 0 on the boundary; ghosts of wide stencils by odd reflection */
  MG_BOUNDARY_PERIODIC = 1   /* [0,1]^2 periodic (Sec. 2.2): stencils and transfers wrap modulo
                                each level's lattice; coarsening continues to a single node */
} mg_boundary;

typedef struct {
  int32_t n;     /* cells per side, power of two */
  double length; /* side of the square domain [0, length]^2, h = length / n; 0 means 1 (the
                    paper's unit square); negative or non-finite: MG_ERR_INVALID */
} mg_grid;

typedef struct {
  double omega;        /* relaxation parameter (default 1.0) */
  int32_t nu1, nu2;    /* pre- and post-smoothing sweeps (default 1, 1) */
  int32_t gamma;       /* 1 = V cycle, 2 = W cycle, 3 = "Wn" cycle: 2 coarse cycles on
                          levels 0 and 1, 1 below (Sec. 4.4) (default 1) */
  int32_t smoother;    /* mg_smoother (default MG_SMOOTH_REDBLACK) */
  int32_t n_min;       /* coarsest axis grid cells per side: a power of two, 2 <= n_min <= n / 2
                          (default 2: one unknown, solved by one division; periodic
                          hierarchies go on to one node, N_l = 1, and accept only 2).
                          n_min > 2 (Dirichlet): the coarsest level's (n_min - 1)^2 unknowns
                          are solved exactly (Algorithm "MG", Sec. 2.2) by a dense factor
                          formed at set-up: Cholesky A = L L^T by columns, G = L^-1 by rows,
                          then x = G^T (G d), every sum in a fixed order (k ascending from
                          the first product), so the iterates are reproducible bit for bit */
  int32_t max_levels;  /* 0 = no limit; otherwise at least 2 (Dirichlet only): the hierarchy
                          stops after that many levels and its coarsest level (axis or
                          rotated, at most 1024 unknowns, else MG_ERR_UNSUPPORTED) takes the
                          dense solve */
  int32_t precision;   /* mg_precision (default MG_PREC_FP64) */
  int32_t fma_contract;/* 0 = separate rounding of every product (default), 1 = FMA allowed */
  int32_t inner_cycles;/* mixed precision: FP32 cycles per refinement step (default 1: FP32
                          rounding caps a step's reduction near 5e-4, so more cycles per
                          step cost more than extra steps) */
  int32_t tail_unknowns;/* the smallest levels run inside one kernel: 0 = built-in default (the
                           levels whose arrays fit a small budget live in one block's shared
                           memory), > 0 = levels (below the finest) with at most this many
                           unknowns run in one thread-block-cluster kernel, -1 = never */
  int32_t tail_ctas;   /* CTAs of that cluster (1..16); 0 = largest the device schedules */
  int32_t sweep_kernel;/* red-black sweeps: 0 = auto (mixed precision: large FP32 axis levels with a
                          5- or 9-point cross stencil run TMA-staged shared-memory tile kernels,
                          nu1 sweeps from zero in one kernel, the residual fused with the
                          red-black restriction, one kernel per post-smoothing sweep; other
                          levels two half-sweep kernels), 1 = half-sweep kernels only, 2 = one
                          shared-memory tile kernel per sweep; every choice gives the same bits */
  int32_t bf16_levels; /* mixed precision, storage trial: values stored on the k finest FP32
                          inner levels are rounded to bfloat16 (0 = off, at most 4; the
                          arrays stay FP32, so this measures accuracy, not bandwidth) */
  int32_t boundary;    /* mg_boundary (default MG_BOUNDARY_DIRICHLET). Periodic is not
                          available with sweep_kernel = 2 or the batch API (MG_ERR_UNSUPPORTED) */
  int32_t transfer_order; /* 2 (default): Eq. (transfer_2d) / (transfer_r2); 4: cubic
                          interpolation and its adjoint restriction, the pair Eq. (interp_2d4o) /
                          (restr_2d4o) (App. A), standard coarsening only (MG_ERR_UNSUPPORTED
                          otherwise, and with the batch API). Ghost coarse nodes beyond the
                          boundary are odd reflections (Dirichlet) or wrap (periodic). Galerkin
                          coefficients over cubic transfers need more than 53 bits from the
                          fourth coarse level on: the recursion is done exactly and each level
                          rounded once to FP64 */
  int32_t dirichlet_data; /* 0 (default): homogeneous Dirichlet data, the boundary entries of u
                          are set to zero; 1: the boundary entries of u hold the data g of
                          B u = g (Sec. 2.1) and are kept (second order, Dirichlet boundary
                          only; MG_ERR_UNSUPPORTED otherwise) */
  /* Device memory of the handle's buffers (default NULL, NULL: cudaMalloc / cudaFree),
     e.g. a framework's caching allocator. Both or neither must be set. dev_alloc returns
     NULL on failure (MG_ERR_OOM); memory must be usable from any stream of the current
     device. mg_destroy synchronises the device before handing buffers to dev_free. The
     callbacks run inside mg_setup, mg_solve_host (its first call) and mg_destroy. */
  void* (*dev_alloc)(size_t bytes, void* ctx);
  void (*dev_free)(void* ptr, void* ctx);
  void* alloc_ctx;
} mg_options;

typedef struct mg_handle mg_handle;

typedef struct {
  int32_t kind;     /* 0 = axis grid, 1 = rotated grid (black points of an axis grid) */
  int32_t n;        /* cells per side of the lattice the level's points live on */
  int32_t rows;     /* storage rows (n + 1) */
  int32_t cols;     /* used storage columns: n + 1 (axis) or n/2 + 1 (rotated) */
  int32_t pitch;    /* elements between rows */
  int32_t unknowns; /* unknowns of the level */
  int32_t nterms;   /* interior stencil size */
  int32_t periodic; /* 1: unknowns are the nodes 0 <= i, j < n; 0: interior nodes 0 < i, j < n */
} mg_level_info;
/* Storage of a level: a rows x pitch array of the level's precision. Axis
   grid: element [j*pitch + i] is lattice node (i, j). Rotated grid: only nodes
   with i + j even exist; node (i, j) is element [j*pitch + (i >> 1)]. */

/* Fill *opt with the defaults listed in mg_options. */
void mg_default_options(mg_options* opt);

/* Build a hierarchy (Sec. 2.2 components 1-4 for the chosen coarsening and
   coarse operators). order is 2 (Eq. L_h_2), 4 (Eq. L_h_2d_4o) or 6 (Eq. LhOrder6,
   the 13-point cross (-2, 27, -270, 980, -270, 27, -2) / (180 h^2); the printed right
   arm's missing separator read as "27, -2"); for orders 4 and 6 the coarse operators
   derive from L_h^(2) except MG_OP_GALERKIN_TRUE_HIGH. opt may be
   NULL (defaults). On success *out owns device memory until mg_destroy.
   Errors: MG_ERR_INVALID (n not a power of two in [4, 16384], bad enum, out NULL),
   MG_ERR_UNSUPPORTED, MG_ERR_OOM, MG_ERR_CUDA. */
mg_status mg_setup(const mg_grid* grid, int order, mg_coarsening coarsening,
                   mg_coarse_op coarse_op, const mg_options* opt, mg_handle** out);

/* One gamma-cycle (Algorithm "MG" of Sec. 2.2 with maxIters = 1) on device
   arrays u (in/out) and f. If rel_res_out is not NULL the stream is
   synchronised and the relative residual after the cycle is stored there.
   Precision MG_PREC_MIXED_FP32: one refinement step (FP64 residual, inner FP32
   cycles, FP64 update). */
mg_status mg_cycle(mg_handle* h, double* u, const double* f, double* rel_res_out, void* stream);

/* Cycle until the relative residual is below rtol or max_cycles cycles ran
   (the while-test of Algorithm "MG", read as "repeat while above tol").
   history_out (may be NULL) receives max_cycles + 1 doubles: entry 0 is the
   initial relative residual, entry k the one after cycle k; entries after the
   last cycle are left unchanged. cycles_out (may be NULL) receives the number
   of cycles run. Returns MG_ERR_NOT_CONVERGED if rtol was not reached,
   MG_ERR_NONFINITE on a NaN/Inf residual, MG_ERR_INVALID if f is zero. */
mg_status mg_solve(mg_handle* h, double* u, const double* f, double rtol, int max_cycles,
                   int* cycles_out, double* history_out, void* stream);

/* mg_solve with u and f in HOST memory ((N+1) x (N+1) doubles, the layout of the
   device arrays above): copies f and u to device arrays the handle owns (allocated
   with cudaMalloc on the first call, 2 (N+1)^2 doubles, freed by mg_destroy), runs
   mg_solve on them, copies the new u back and synchronises the stream before
   returning. The copies are asynchronous only from pinned (page-locked) host memory;
   from pageable memory they are staged by the CUDA runtime. Same results, statuses and
   history as mg_solve; on statuses other than MG_OK and MG_ERR_NOT_CONVERGED u_host is
   left unchanged. */
mg_status mg_solve_host(mg_handle* h, double* u_host, const double* f_host, double rtol, int max_cycles,
                        int* cycles_out, double* history_out, void* stream);

/* Release every buffer of the handle (NULL is accepted). */
mg_status mg_destroy(mg_handle* h);

/* Static text for a status code. */
const char* mg_status_string(mg_status s);

/* Device bytes mg_setup would allocate for these arguments (0 if invalid). */
size_t mg_workspace_bytes(const mg_grid* grid, int order, mg_coarsening coarsening,
                          mg_coarse_op coarse_op, const mg_options* opt);

/* Number of levels (finest = 0, coarsest = mg_num_levels - 1), or -1. */
int mg_num_levels(const mg_handle* h);

/* Layout of level `level`. */
mg_status mg_get_level_info(const mg_handle* h, int level, mg_level_info* out);

/* ---- single steps of the cycle on caller buffers in a level's storage ------
   All pointers are device pointers in the FP64 storage of the named level(s)
   (mg_get_level_info); boundary entries are read as zero and never written. */

/* out = L_l u on interior nodes. */
mg_status mg_level_apply(mg_handle* h, int level, const double* u, double* out, void* stream);
/* d = f - L_l u on interior nodes (Algorithm "MG", residual step). */
mg_status mg_level_residual(mg_handle* h, int level, const double* u, const double* f,
                            double* d, void* stream);
/* `sweeps` smoothing sweeps in place on u (red-black: red half-sweep then black). */
mg_status mg_level_smooth(mg_handle* h, int level, double* u, const double* f, int sweeps,
                          void* stream);
/* f_coarse = R d_fine, R from level `level` to level + 1 (Eq. transfer_r2 / transfer_2d). */
mg_status mg_level_restrict(mg_handle* h, int level, const double* d_fine, double* f_coarse,
                            void* stream);
/* u_fine += P v_coarse, P from level + 1 to level `level`. */
mg_status mg_level_prolong_add(mg_handle* h, int level, double* u_fine, const double* v_coarse,
                               void* stream);

/* ---- batched solves (many independent problems) -------------------------------
   Algorithm "MG" (Sec. 2.2) run on many grids at once; the paper has no batched form.
   A batch advances many handles together by a level-synchronous schedule: each step
   of the V-cycle (a half-sweep, residual, restriction, interpolation, ... of level l)
   is ONE kernel launch covering level l of every problem that has it, with blocks
   mapped to (problem, tile) pairs; problems that have converged are masked by device
   flags, so the inner cycle is one CUDA graph for the whole batch. Per-problem
   results are bitwise those of mg_solve on each handle alone (same operations per
   node, same order). All handles must share precision, nu1, nu2, fma_contract and
   (mixed precision) inner_cycles; gamma must be 1, the smoother red-black and the
   boundary Dirichlet (MG_ERR_UNSUPPORTED otherwise); a handle may appear only once
   (MG_ERR_INVALID). mg_batch_create also autotunes, per level, the rows
   per thread of the step kernels by timing them (CUDA events), so create the batch
   once and reuse it. The batch keeps pointers to the handles: destroy the batch
   before them.

   Hybrid schedule: problems whose grid side N is at least solo_min_n are not in the
   level-synchronous schedule. Each is solved by mg_solve on its own handle, on one of
   `workers` internal non-blocking streams, each driven by a host thread that takes the
   next unsolved problem, largest first. Meanwhile the calling thread runs the
   level-synchronous schedule of the other problems. A large problem's own mg_solve
   runs its single-problem kernels (TMA tiles, fused coarse tail); a small problem's
   levels leave most SMs idle alone, which the level-synchronous steps fill. The
   caller's stream waits for all of it. Results stay bitwise those of mg_solve alone.
   mg_batch_options (opt may be NULL: the defaults):
     solo_min_n  0: default 1024; a value above 16384 puts every problem in the
                 level-synchronous schedule; negative: MG_ERR_INVALID.
     workers     0: default 12 (at most the number of solo problems); 1..64. */
typedef struct mg_batch mg_batch;
typedef struct {
  int solo_min_n;
  int workers;
} mg_batch_options;
mg_status mg_batch_create_ex(mg_handle* const* handles, int count, const mg_batch_options* opt, mg_batch** out);
/* mg_batch_create_ex with the default options. */
mg_status mg_batch_create(mg_handle* const* handles, int count, mg_batch** out);
/* Solve problem p: u[p], f[p] device arrays of handle p's finest level. Per problem:
   cycles (refinement steps for mixed precision) in cycles_out[p] and the final
   relative residual in rel_res_out[p] (either may be NULL). Returns
   MG_ERR_NOT_CONVERGED if any problem missed rtol within max_cycles. With solo
   problems, the call starts up to `workers` host threads and joins them before it
   returns; the first error wins (the level-synchronous part's, then the solo problems'
   in index order). After an error other than MG_ERR_NOT_CONVERGED the outputs of the
   failed problems carry no meaning. One call at a time per batch. */
mg_status mg_batch_solve(mg_batch* b, double* const* u, const double* const* f, double rtol, int max_cycles,
                         int* cycles_out, double* rel_res_out, void* stream);
mg_status mg_batch_destroy(mg_batch* b);
/* Kernels launched through the batch so far, solo solves included (graph launches
   count their kernels). */
mg_status mg_batch_get_launches(const mg_batch* b, int64_t* launches);
/* Convenience: create a batch, solve once, destroy it. */
mg_status mg_solve_batched(mg_handle* const* handles, double* const* u, const double* const* f, int count,
                           double rtol, int max_cycles, int* cycles_out, double* rel_res_out, void* stream);

/* ---- relative residual without device allocation ----------------------------
   The paper has no counterpart to this call; it serves callers that must not
   allocate device memory at the point where they need a residual norm: loops that
   cannot afford the implicit device synchronisation of cudaMalloc / cudaFree, or hosts
   that fix the library's memory at set-up (a budget, or an arena they manage).
   Writes ||f - L_h u||_2 / ||f||_2 over the finest level's interior nodes (same
   evaluation order as mg_cycle's rel_res_out, partial sums added in a different
   fixed order) to the DEVICE double *rel_res_dev, asynchronously on `stream`.
   u and f are device arrays of the finest level (as for mg_cycle); u's boundary is
   read as stored. It calls no allocator: the reduction's partial sums live in one
   32 KB device array inside the library (2 x 2048 doubles), which every GPU that
   loads the library holds until the process exits. The first call on a device looks
   up that array's device address (and may make the CUDA runtime load the library's
   device code), so make the first call on each device before any stream capture. The
   looked-up address is kept for the life of the process: after a cudaDeviceReset, do not
   call it again on that device.
   All calls share the array and each call overwrites the partials it reads, so no
   state carries over; calls whose work overlaps on the GPU (different streams, or
   several host threads) race on the array and must be serialised by the caller.
   Returns MG_ERR_UNSUPPORTED if the finest grid needs more than 2048 partial sums
   per row of tiles (N + 1 > 65536 columns; unreachable for N <= 16384),
   MG_ERR_INVALID for NULL arguments, MG_ERR_CUDA if a launch fails. */
mg_status mg_rel_residual_static(mg_handle* h, const double* u, const double* f, double* rel_res_dev,
                                 void* stream);

/* ---- instrumentation --------------------------------------------------------
   Counters of kernel launches and cycles made through the handle, and optional
   CUDA-event timing of the finest level's kernels (recorded on the stream the
   kernels are launched on). Not part of the paper's method. */
typedef struct {
  int64_t launches; /* kernels launched by the library since the last reset */
  int64_t cycles;   /* multigrid cycles run since the last reset */
} mg_counters;

typedef enum {
  MG_KERNEL_SMOOTH = 0,   /* finest-level smoothing sweeps */
  MG_KERNEL_RESIDUAL = 1, /* finest-level residual */
  MG_KERNEL_RESTRICT = 2, /* restriction from the finest level */
  MG_KERNEL_PROLONG = 3,  /* interpolation + correction into the finest level */
  MG_KERNEL_NORM = 4,     /* residual-norm reduction */
  MG_KERNEL_CLASSES = 5
} mg_kernel_class;

mg_status mg_get_counters(const mg_handle* h, mg_counters* out);
mg_status mg_reset_counters(mg_handle* h);
/* enable = 1: record a CUDA event pair around every finest-level launch; 2: around
   every launch of every level (kernel class k of level l is read as k + 5 l; a tail
   kernel counts as level l's MG_KERNEL_SMOOTH); 0: off. Timed runs launch eagerly
   (no CUDA graph). */
mg_status mg_set_timing(mg_handle* h, int enable);
/* Total device milliseconds and launch count of a kernel class since timing was
   enabled or last read (waits for the recorded events; resets the class). */
mg_status mg_get_timing(mg_handle* h, int kernel_class, double* total_ms, int64_t* launches);

#ifdef __cplusplus
}
#endif

#endif /* NSMG_H */
