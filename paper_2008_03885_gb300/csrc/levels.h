// Internal types shared by the host hierarchy code and the CUDA kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace nsmg {

constexpr int kMaxTerms = 128;  // largest interior stencil a level may carry (cubic-transfer
                                // Galerkin stencils reach 11 x 11 = 121 terms)

enum Kind : int32_t { kAxis = 0, kRot = 1 };

// Grid transfer between level l (fine) and l + 1 (coarse).
enum Transfer : int32_t {
  kRbAxisToRot = 0,  // axis fine grid -> its black points (same lattice)
  kRbRotToAxis = 1,  // rotated fine grid -> points with i, j even (lattice n/2)
  kStandard = 2,     // axis n -> axis n/2, bilinear / full weighting
  kStandardCubic = 3 // axis n -> axis n/2, cubic interpolation and its adjoint (R = 1/4 P^T)
};

// A merged boundary-class term: coefficient and lattice offset in one aligned 16-byte
// record, so that one vector load fetches it. The first term of each group of equal
// coefficients (see LevelDev::gmask) carries kTermStart added to dx.
constexpr int32_t kTermStart = 1 << 20;
template <typename T>
struct __align__(16) ClassTerm {
  T c;
  int32_t dx, dy;
};

// Device-resident description of one level in precision T.
//
// Points live on an integer lattice (i, j), 0 <= i, j <= n. Axis levels hold every
// node; rotated levels hold nodes with i + j even and store node (i, j) at column
// i >> 1. Dirichlet (per = 0): interior nodes 0 < i, j < n are the unknowns and
// boundary entries of every array are 0. Periodic (per = 1): nodes 0 <= i, j < n are
// the unknowns (node n is node 0); row and column n are never read.
//
// The operator is a constant stencil (dx, dy, c) for "fast"
// nodes, rx <= i <= n - per - rx (the same for j with ry): their stencil reaches no
// ghost (Dirichlet) and does not wrap (periodic). Other nodes use a per-class merged
// term list: the stencil folded by odd reflection at the boundary lines with
// boundary columns dropped (Dirichlet) or wrapped modulo n (periodic; the stored
// offsets are the wrapped ones), duplicate columns summed, sorted by (dy, dx), which
// is the storage (column) order. A class is (cx, cy):
//   small levels: cx = i, cy = j (table (n+1) x (n+1));
//   otherwise: cx = i for i < rx, 2 rx - (n - per - i) for i > n - per - rx, rx in
//   between (single coordinates at both edges, so every class has one term list).
template <typename T>
struct LevelDev {
  int32_t kind, n, rows, cols, pitch;
  int32_t nt, rx, ry;
  int32_t small, clsw;
  T wd;                       // omega / a_pp at fast nodes
  T c[kMaxTerms];             // fast-node coefficients, in evaluation order: groups of equal
                              // coefficient (ordered by their first term in (dy, dx) order),
                              // each group's terms in (dy, dx) order
  uint32_t gmask[kMaxTerms / 32];  // bit k: fast term k starts a group
  int32_t delta[2][kMaxTerms];  // storage offsets of the fast terms for i even / odd
  int32_t sdx[2][kMaxTerms];    // storage-column shift of the fast terms for i even / odd
  int32_t sdy[kMaxTerms];       // row shift of the fast terms
  const int2* cls;            // per class: (first term, term count)
  const T* cls_wd;            // per class: omega / a_pp
  const ClassTerm<T>* terms;  // merged terms of every class
  int32_t bf16;  // FP32 inner levels: round every stored value to bfloat16 (storage trial)
  int32_t per;   // 1: periodic level (see above)
  int32_t lo;    // first unknown index: 1 - per
  int32_t fxe, fye;  // last fast-node i and j: n - per - rx, n - per - ry
};

}  // namespace nsmg
