// Multigrid kernels for sm_103a: stencil application with boundary classes,
// red-black and Jacobi relaxation, residual, restriction, interpolation with
// correction, coarsest solve, and a deterministic residual-norm reduction.
//
// Evaluation order (EXACT = true): an operator row is sum_g c_g * (x_g1 + x_g2 + ...)
// over its groups of equal coefficient (groups ordered by their first term in (dy, dx)
// order, each group's terms in (dy, dx) order), every sum left to right and every
// product and sum rounded separately (__dmul_rn / __dadd_rn keep nvcc from contracting
// them into FMAs); grid transfers sum their products in the order of their term lists.
// EXACT = false lets products fuse into FMAs (one per term, in the same term order).
#include <algorithm>
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cstdio>

#include "kernels.h"
#include "device.cuh"

namespace nsmg {
namespace {

template <typename T, bool EXACT, int NT, bool PER>
__global__ void __launch_bounds__(kBX * kBY, MinBlocks<T>::value) k_half_sweep_nt(const LevelDev<T>* __restrict__ Lp, const T* __restrict__ uin,
                                const T* __restrict__ f, T* __restrict__ uout, int red) {
  constexpr int kRows = RowsPer<T>::value;
  const LevelDev<T>& L = *Lp;
  T c[NT];
  int d0[NT], d1[NT];
#pragma unroll
  for (int k = 0; k < NT; ++k) {
    c[k] = L.c[k];
    d0[k] = L.delta[0][k];
    d1[k] = L.delta[1][k];
  }
  const T wd = L.wd;
  const int n = L.n;
  constexpr int lo = PER ? 0 : 1;
  const int jb = blockIdx.y * (kBY * kRows) + threadIdx.y;
  // Prefetch the thread's u and f lines of all its rows into L2 before the first row's
  // loads. Measured on GB300 at 4097^2: FP32 axis half-sweep 59.5 -> 55.3 us (order 4),
  // 52.3 -> 45.8 us (order 2); FP64 rotated 178 -> 173 us; no gain (or a loss) for the
  // other two combinations, which skip it.
  if ((sizeof(T) == 4) == (L.kind == kAxis)) {
    const int col = L.kind == kAxis ? min(2 * (int)(blockIdx.x * kBX + threadIdx.x), n)
                                    : min((int)(blockIdx.x * kBX + threadIdx.x), L.cols - 1);
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const int64_t at = (int64_t)min(jb + r * kBY, L.rows - 1) * L.pitch + col;
      prefetch_l2(uin + at);
      prefetch_l2(f + at);
    }
  }
  if (L.kind == kAxis) {
    const int i0 = 2 * (blockIdx.x * kBX + threadIdx.x);
    if (i0 > n) return;
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const int j = jb + r * kBY;
      if (j < lo || j >= n) continue;
      const int i = (((i0 + j) & 1) == red) ? i0 : i0 + 1;
      const int ic = 2 * i0 + 1 - i;
      const int64_t row = (int64_t)j * L.pitch;
      if (ic >= lo && ic < n) uout[row + ic] = uin[row + ic];
      if (i < lo || i >= n) continue;
      const int64_t at = row + i;
      uout[at] = rnd(L, fast_node_c<PER>(L, i, j) ? relax_fast<T, EXACT, NT>(c, d0, wd, uin, f, at)
                                                  : relax_value<T, EXACT, 1>(L, uin, f, i, j, at));
    }
  } else {
    const int q = blockIdx.x * kBX + threadIdx.x;
    if (q >= L.cols) return;
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const int j = jb + r * kBY;
      if (j < lo || j >= n) continue;
      const int i = 2 * q + (j & 1);
      if (i < lo || i >= n) continue;
      const int64_t at = (int64_t)j * L.pitch + q;
      if ((i & 1) != red) {
        uout[at] = uin[at];
        continue;
      }
      uout[at] = rnd(L, fast_node_c<PER>(L, i, j) ? relax_fast<T, EXACT, NT>(c, (i & 1) ? d1 : d0, wd, uin, f, at)
                                                  : relax_value<T, EXACT, 1>(L, uin, f, i, j, at));
    }
  }
}

template <typename T, bool EXACT, int NT, bool PER>
__global__ void __launch_bounds__(kBX * kBY, MinBlocks<T>::value) k_residual_nt(const LevelDev<T>* __restrict__ Lp, const T* __restrict__ u,
                              const T* __restrict__ f, T* __restrict__ d) {
  constexpr int kRows = RowsPer<T>::value;
  const LevelDev<T>& L = *Lp;
  T c[NT];
  int d0[NT], d1[NT];
#pragma unroll
  for (int k = 0; k < NT; ++k) {
    c[k] = L.c[k];
    d0[k] = L.delta[0][k];
    d1[k] = L.delta[1][k];
  }
  const int n = L.n;
  constexpr int lo = PER ? 0 : 1;
  const int q = blockIdx.x * kBX + threadIdx.x;
  if (q >= L.cols) return;
  const int jb = blockIdx.y * (kBY * kRows) + threadIdx.y;
  // Same L2 prefetch as the half-sweeps: FP32 level-0 residual 120 -> 103 us at 4097^2
  // (order 4); FP64 (bound by the FP64 pipe) unchanged, so it skips it.
  if (sizeof(T) == 4) {
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const int64_t at = (int64_t)min(jb + r * kBY, L.rows - 1) * L.pitch + q;
      prefetch_l2(u + at);
      prefetch_l2(f + at);
    }
  }
#pragma unroll
  for (int r = 0; r < kRows; ++r) {
    const int j = jb + r * kBY;
    if (j < lo || j >= n) continue;
    const int i = L.kind == kRot ? 2 * q + (j & 1) : q;
    if (i < lo || i >= n) continue;
    const int64_t at = (int64_t)j * L.pitch + q;
    const T s = fast_node_c<PER>(L, i, j) ? apply_fast<T, EXACT, NT>(c, (L.kind == kRot && (i & 1)) ? d1 : d0, u, at)
                                          : apply_at<T, EXACT, 1>(L, u, i, j, at, nullptr);
    d[at] = rnd(L, Arith<T>::sub(f[at], s));
  }
}

// Wide stencils (any size): one node per thread; the interior stencil's
// coefficients and storage offsets are staged in shared memory once per block.
template <typename T>
struct StencilSmem {
  T c[kMaxTerms];
  int d[2][kMaxTerms];
  uint32_t gm[kMaxTerms / 32];
};

template <typename T>
__device__ __forceinline__ void stage_stencil(const LevelDev<T>& L, StencilSmem<T>& sm) {
  for (int k = threadIdx.y * blockDim.x + threadIdx.x; k < L.nt; k += blockDim.x * blockDim.y) {
    sm.c[k] = L.c[k];
    sm.d[0][k] = L.delta[0][k];
    sm.d[1][k] = L.delta[1][k];
  }
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  if (t < kMaxTerms / 32) sm.gm[t] = L.gmask[t];
  __syncthreads();
}

// U: unroll factor of the term loop (its loads then run ahead of the ordered sum).
template <typename T, bool EXACT, int U = 4>
__device__ __forceinline__ T apply_smem(const StencilSmem<T>& sm, int nt, int par, const T* __restrict__ u, int64_t at) {
  const int* dl = sm.d[par];
  RowSum<T, EXACT> acc;
#pragma unroll U
  for (int k = 0; k < nt; ++k) acc.add(sm.c[k], u[at + dl[k]], gbit(sm.gm, k));
  return acc.value();
}

// Wide-stencil kernels. DEEP (FP32, levels below kGenDeepRows rows): the term loop
// unrolled 8 deep with 48 registers (5 blocks per SM) so that more of a node's loads are
// in flight; on those small, latency-bound levels this measured faster (4097^2 mixed
// solve 16.5 -> 15.5 ms), on larger FP32 levels slower (2049^2: 36 vs 33 us per half-sweep).
template <typename T, bool DEEP>
struct GenCfg {
  static constexpr bool deep = DEEP && sizeof(T) == 4;
  static constexpr int min_blocks = deep ? 5 : MinBlocks<T>::value;
  static constexpr int unroll = deep ? 8 : 4;
};
constexpr int kGenDeepRows = 2048;

template <typename T, bool EXACT, bool DEEP>
__global__ void __launch_bounds__(kBX * kBY, GenCfg<T, DEEP>::min_blocks) k_half_sweep_gen(const LevelDev<T>* __restrict__ Lp, const T* __restrict__ uin,
                                 const T* __restrict__ f, T* __restrict__ uout, int red) {
  const LevelDev<T>& L = *Lp;
  __shared__ StencilSmem<T> sm;
  stage_stencil(L, sm);
  int i, j;
  if (L.kind == kAxis) {
    const int i0 = 2 * (blockIdx.x * kBX + threadIdx.x);
    j = blockIdx.y * blockDim.y + threadIdx.y;
    const int lo = L.lo;
    if (j < lo || j >= L.n || i0 > L.n) return;
    i = (((i0 + j) & 1) == red) ? i0 : i0 + 1;
    const int ic = 2 * i0 + 1 - i;
    if (ic >= lo && ic < L.n) {
      const int64_t ac = sidx(L, ic, j);
      uout[ac] = uin[ac];
    }
    if (i < lo || i >= L.n) return;
  } else {
    if (!thread_node(L, i, j) || !interior(L, i, j)) return;
    if (is_red(L, i, j) != red) {
      const int64_t at = sidx(L, i, j);
      uout[at] = uin[at];
      return;
    }
  }
  const int64_t at = sidx(L, i, j);
  if (fast_node(L, i, j)) {
    const T r = Arith<T>::sub(f[at], apply_smem<T, EXACT, GenCfg<T, DEEP>::unroll>(sm, L.nt, L.kind == kRot ? (i & 1) : 0,
                                                                                 uin, at));
    const T wd = L.wd;
    uout[at] = rnd(L, EXACT ? Arith<T>::add(uin[at], Arith<T>::mul(r, wd)) : Arith<T>::fma(r, wd, uin[at]));
  } else {
    uout[at] = rnd(L, relax_value<T, EXACT>(L, uin, f, i, j, at));
  }
}

template <typename T, bool EXACT, bool DEEP>
__global__ void __launch_bounds__(kBX * kBY, GenCfg<T, DEEP>::min_blocks) k_residual_gen(const LevelDev<T>* __restrict__ Lp, const T* __restrict__ u,
                               const T* __restrict__ f, T* __restrict__ d) {
  const LevelDev<T>& L = *Lp;
  __shared__ StencilSmem<T> sm;
  stage_stencil(L, sm);
  int i, j;
  if (!thread_node(L, i, j) || !interior(L, i, j)) return;
  const int64_t at = sidx(L, i, j);
  const T s = fast_node(L, i, j) ? apply_smem<T, EXACT, GenCfg<T, DEEP>::unroll>(sm, L.nt, L.kind == kRot ? (i & 1) : 0, u, at)
                                 : apply_at<T, EXACT>(L, u, i, j, at, nullptr);
  d[at] = rnd(L, Arith<T>::sub(f[at], s));
}

// ---- fused red-black sweep on a shared-memory tile ---------------------------
// One kernel does the red then the black half-sweep of a kFTW x kFTH tile of storage
// elements: the tile plus a halo of two relaxation reaches (2 rq columns, 2 ry rows)
// of u and f is staged in shared memory, red nodes are relaxed on the tile plus one
// reach (so every black node of the tile sees updated red neighbours), then black
// nodes of the tile. Arithmetic per node is exactly relax_value's. Threads are a
// 32 x 8 grid walking the shared arrays row by row (coalesced global loads).
constexpr int kFTW = 64, kFTH = 32;

// Level scalars the tile kernel needs, held in registers.
struct TileGeom {
  int kind, n, rows, cols, pitch, rx, ry, nt;
};

template <typename T, bool EXACT, int NT>
__device__ __forceinline__ T relax_tile(const LevelDev<T>& L, const TileGeom& G, T wdf, const T* __restrict__ su,
                                        const T* __restrict__ sf, const T* sc, const int* soff, int e, int i, int j,
                                        int q0, int j0, int SW) {
  T wd;
  RowSum<T, EXACT> acc;
  if (i >= G.rx && i <= G.n - G.rx && j >= G.ry && j <= G.n - G.ry) {
    if (NT > 0) {
#pragma unroll
      for (int k = 0; k < NT; ++k) acc.add(sc[k], su[e + soff[k]], gbit(L.gmask, k));
    } else {
#pragma unroll 4
      for (int k = 0; k < G.nt; ++k) acc.add(sc[k], su[e + soff[k]], gbit(L.gmask, k));
    }
    wd = wdf;
  } else {
    const int cl = class_of(L, i, j);
    const int2 ce = L.cls[cl];
    const ClassTerm<T>* tt = L.terms + ce.x;
#pragma unroll 4
    for (int k = 0; k < ce.y; ++k) {
      const Term<T> t = load_term(tt + k);
      const int ti = i + t.dx, tj = j + t.dy;
      const int tq = G.kind == kRot ? (ti >> 1) : ti;
      acc.add(t.c, su[(tj - j0) * SW + (tq - q0)], t.start);
    }
    wd = L.cls_wd[cl];
  }
  const T s = acc.value();
  const T r = Arith<T>::sub(sf[e], s);
  return EXACT ? Arith<T>::add(su[e], Arith<T>::mul(r, wd)) : Arith<T>::fma(r, wd, su[e]);
}

template <typename T, bool EXACT, int NT>
__global__ void __launch_bounds__(kBX * kBY)
    k_sweep_fused(const LevelDev<T>* __restrict__ Lp, const T* __restrict__ uin, const T* __restrict__ f,
                  T* __restrict__ uout, int rq, int ry) {
  extern __shared__ __align__(16) unsigned char fused_smem[];
  __shared__ T sc[kMaxTerms];
  __shared__ int soff[2][kMaxTerms];
  const LevelDev<T>& L = *Lp;
  const TileGeom G{L.kind, L.n, L.rows, L.cols, L.pitch, L.rx, L.ry, L.nt};
  const T wdf = L.wd;
  const int hx = 2 * rq, hy = 2 * ry;
  const int SW = kFTW + 2 * hx, SH = kFTH + 2 * hy, SN = SW * SH;
  T* su = reinterpret_cast<T*>(fused_smem);
  T* sf = su + SN;
  T* st = sf + SN;
  const int q0 = blockIdx.x * kFTW - hx;  // storage coordinates of shared element 0
  const int j0 = blockIdx.y * kFTH - hy;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kBX + tx;
  if (tid < G.nt) {
    sc[tid] = L.c[tid];
    soff[0][tid] = L.sdy[tid] * SW + L.sdx[0][tid];
    soff[1][tid] = L.sdy[tid] * SW + L.sdx[1][tid];
  }
  for (int lj = ty; lj < SH; lj += kBY) {
    const int gj = j0 + lj;
    const bool rowok = gj >= 0 && gj < G.rows;
    for (int lq = tx; lq < SW; lq += kBX) {
      const int gq = q0 + lq;
      T vu = T(0), vf = T(0);
      if (rowok && gq >= 0 && gq < G.pitch) {
        const int64_t at = (int64_t)gj * G.pitch + gq;
        vu = uin[at];
        vf = f[at];
      }
      su[lj * SW + lq] = vu;
      sf[lj * SW + lq] = vf;
    }
  }
  __syncthreads();
  const bool rot = G.kind == kRot;
  // Colour-mapped walks over a shared-memory window [lq_lo, lq_hi) x [lj_lo, lj_hi):
  // axis grids hold one colour on every other column of a row (lanes take stride 2),
  // rotated grids one colour per row (threads take every other row).
  auto walk = [&](int lq_lo, int lq_hi, int lj_lo, int lj_hi, bool want_red, auto&& body) {
    if (rot) {
      // red rows: j odd
      int lj = lj_lo + ((((j0 + lj_lo) & 1) != (want_red ? 1 : 0)) ? 1 : 0);
      for (lj += 2 * ty; lj < lj_hi; lj += 2 * kBY) {
        const int j = j0 + lj;
        if (j <= 0 || j >= G.n) continue;
        for (int lq = lq_lo + tx; lq < lq_hi; lq += kBX) {
          const int gq = q0 + lq;
          if (gq < 0 || gq >= G.cols) continue;
          const int i = 2 * gq + (j & 1);
          if (i <= 0 || i >= G.n) continue;
          body(lj * SW + lq, i, j, gq);
        }
      }
    } else {
      for (int lj = lj_lo + ty; lj < lj_hi; lj += kBY) {
        const int j = j0 + lj;
        if (j <= 0 || j >= G.n) continue;
        // red: (gq + j) odd
        const int want = want_red ? 1 : 0;
        int lq = lq_lo + ((((q0 + lq_lo + j) & 1) != want) ? 1 : 0);
        for (lq += 2 * tx; lq < lq_hi; lq += 2 * kBX) {
          const int gq = q0 + lq;
          if (gq <= 0 || gq >= G.n) continue;
          body(lj * SW + lq, gq, j, gq);
        }
      }
    }
  };
  const int* soff_r = soff[rot ? 1 : 0];  // red nodes of a rotated grid have i odd
  const int* soff_b = soff[0];            // black nodes of a rotated grid have i even
  // red half-sweep on the tile plus one reach (new values into st)
  walk(hx - rq, hx + kFTW + rq, hy - ry, hy + kFTH + ry, true, [&](int e, int i, int j, int) {
    st[e] = relax_tile<T, EXACT, NT>(L, G, wdf, su, sf, sc, soff_r, e, i, j, q0, j0, SW);
  });
  __syncthreads();
  walk(hx - rq, hx + kFTW + rq, hy - ry, hy + kFTH + ry, true, [&](int e, int, int, int) { su[e] = st[e]; });
  __syncthreads();
  // tile outputs: red nodes copied from shared memory, black nodes relaxed
  walk(hx, hx + kFTW, hy, hy + kFTH, true, [&](int e, int, int j, int gq) {
    uout[(int64_t)j * G.pitch + gq] = su[e];
  });
  walk(hx, hx + kFTW, hy, hy + kFTH, false, [&](int e, int i, int j, int gq) {
    uout[(int64_t)j * G.pitch + gq] = relax_tile<T, EXACT, NT>(L, G, wdf, su, sf, sc, soff_b, e, i, j, q0, j0, SW);
  });
}

template <typename T, bool EXACT>
__global__ void k_jacobi(const LevelDev<T>* __restrict__ Lp, const T* __restrict__ uin,
                         const T* __restrict__ f, T* __restrict__ uout) {
  const LevelDev<T>& L = *Lp;
  int i, j;
  if (!thread_node(L, i, j) || !interior(L, i, j)) return;
  const int64_t at = sidx(L, i, j);
  T wd;
  const T s = apply_at<T, EXACT>(L, uin, i, j, at, &wd);
  const T r = Arith<T>::sub(f[at], s);
  uout[at] = rnd(L, EXACT ? Arith<T>::add(uin[at], Arith<T>::mul(r, wd)) : Arith<T>::fma(r, wd, uin[at]));
}

template <typename T, bool EXACT>
__global__ void k_apply(const LevelDev<T>* __restrict__ Lp, const T* __restrict__ u,
                        T* __restrict__ out) {
  const LevelDev<T>& L = *Lp;
  int i, j;
  if (!thread_node(L, i, j) || !interior(L, i, j)) return;
  const int64_t at = sidx(L, i, j);
  out[at] = apply_at<T, EXACT>(L, u, i, j, at, nullptr);
}

// Restriction terms (dx, dy) in fine-lattice units, sorted by (dy, dx), with weights.
// Restriction terms of each transfer in the order of the sum: the red-black transfers'
// R = 1/2 P^T (centre 1/2, four neighbours 1/8: axis neighbours from an axis level,
// diagonal ones from a rotated level) and full weighting R = 1/4 P^T for H = 2h
// (Eq. (transfer_r2), Eq. (transfer_2d)). Compile-time functions, so that inside a
// kernel specialised on the transfer every weight is a literal.
__host__ __device__ constexpr int rt_count(int tr) { return tr == kStandard ? 9 : 5; }
__host__ __device__ constexpr int rt_dx(int tr, int k) {
  return tr == kStandard ? k % 3 - 1
         : tr == kRbAxisToRot ? (k >= 1 && k <= 3 ? k - 2 : 0)
                              : (k == 2 ? 0 : (k == 0 || k == 3) ? -1 : 1);
}
__host__ __device__ constexpr int rt_dy(int tr, int k) {
  return tr == kStandard ? k / 3 - 1
         : tr == kRbAxisToRot ? (k == 0 ? -1 : k == 4 ? 1 : 0)
                              : (k < 2 ? -1 : k > 2 ? 1 : 0);
}
__host__ __device__ constexpr double rt_w(int tr, int k) {
  return tr == kStandard ? (rt_dx(tr, k) == 0 ? 2 : 1) * (rt_dy(tr, k) == 0 ? 2 : 1) * 0.0625 : (k == 2 ? 0.5 : 0.125);
}

// Storage position of lattice node (i, j): in the level's global storage, or in the
// compact rows x cols layout of the shared-memory tail.
template <typename T>
__device__ __forceinline__ int smem_idx(const LevelDev<T>& L, int i, int j) {
  return j * L.cols + (L.kind == kRot ? (i >> 1) : i);
}
struct GlobalIdx {
  template <typename T>
  __device__ __forceinline__ int64_t operator()(const LevelDev<T>& L, int i, int j) const { return sidx(L, i, j); }
};
struct SmemIdx {
  template <typename T>
  __device__ __forceinline__ int64_t operator()(const LevelDev<T>& L, int i, int j) const { return smem_idx(L, i, j); }
};

// Periodic transfers: terms (lattice i, j, weight) on level L wrap modulo L.n, are
// ordered by storage position (which is the row-major column order) and terms that
// land on the same node merge by adding their weights (powers of two and their
// small sums, so the merged weight is exact); then the usual ordered sum.
constexpr int kMaxTransferTerms = 25;
template <typename T, bool EXACT, class Idx>
__device__ __forceinline__ T wrapped_sum(const LevelDev<T>& L, int nt, const int* ti, const int* tj, const T* w,
                         const T* __restrict__ x, Idx idx) {
  int64_t pos[kMaxTransferTerms];
  T wt[kMaxTransferTerms];
  int m = 0;
  for (int k = 0; k < nt; ++k) {
    int a = ti[k] % L.n;
    if (a < 0) a += L.n;
    int b = tj[k] % L.n;
    if (b < 0) b += L.n;
    const int64_t p = idx(L, a, b);
    int q = 0;
    while (q < m && pos[q] < p) ++q;
    if (q < m && pos[q] == p) {
      wt[q] = Arith<T>::add(wt[q], w[k]);
      continue;
    }
    for (int r = m; r > q; --r) {
      pos[r] = pos[r - 1];
      wt[r] = wt[r - 1];
    }
    pos[q] = p;
    wt[q] = w[k];
    ++m;
  }
  T s = Arith<T>::mul(wt[0], x[pos[0]]);
  for (int k = 1; k < m; ++k) s = madd<T, EXACT>(s, wt[k], x[pos[k]]);
  return s;
}

// Restriction from a periodic level.
template <typename T, bool EXACT, int TR, class Idx>
__device__ __forceinline__ T restrict_wrapped(const LevelDev<T>& Lf, const T* __restrict__ d, int fi, int fj,
                                              Idx idx) {
  constexpr int nt = rt_count(TR);
  int ti[kMaxTransferTerms], tj[kMaxTransferTerms];
  T w[kMaxTransferTerms];
#pragma unroll
  for (int k = 0; k < nt; ++k) {
    ti[k] = fi + rt_dx(TR, k);
    tj[k] = fj + rt_dy(TR, k);
    w[k] = T(rt_w(TR, k));
  }
  return wrapped_sum<T, EXACT>(Lf, nt, ti, tj, w, d, idx);
}

template <typename T, bool EXACT, int TR, class Idx>
__device__ __forceinline__ T restrict_sum(const LevelDev<T>& Lf, const T* __restrict__ d, int fi, int fj, Idx idx) {
  T s = Arith<T>::mul(T(rt_w(TR, 0)), d[idx(Lf, fi + rt_dx(TR, 0), fj + rt_dy(TR, 0))]);
#pragma unroll
  for (int k = 1; k < rt_count(TR); ++k)
    s = madd<T, EXACT>(s, T(rt_w(TR, k)), d[idx(Lf, fi + rt_dx(TR, k), fj + rt_dy(TR, k))]);
  return s;
}

// Restricted residual at coarse node (i, j) (coarse-level lattice). PER: the levels
// are periodic (a compile-time choice, so that the Dirichlet kernels carry none of
// the wrap-around code).
template <typename T, bool EXACT, bool PER, class Idx = GlobalIdx>
__device__ __forceinline__ T restrict_value(const LevelDev<T>& Lf, int transfer, const T* __restrict__ d,
                                            int i, int j, Idx idx = Idx()) {
  // fine-lattice position of the coarse node
  const int fi = transfer == kRbAxisToRot ? i : 2 * i;
  const int fj = transfer == kRbAxisToRot ? j : 2 * j;
  if (PER) {
    if (transfer == kRbAxisToRot) return restrict_wrapped<T, EXACT, kRbAxisToRot>(Lf, d, fi, fj, idx);
    if (transfer == kRbRotToAxis) return restrict_wrapped<T, EXACT, kRbRotToAxis>(Lf, d, fi, fj, idx);
    return restrict_wrapped<T, EXACT, kStandard>(Lf, d, fi, fj, idx);
  }
  if (transfer == kRbAxisToRot) return restrict_sum<T, EXACT, kRbAxisToRot>(Lf, d, fi, fj, idx);
  if (transfer == kRbRotToAxis) return restrict_sum<T, EXACT, kRbRotToAxis>(Lf, d, fi, fj, idx);
  return restrict_sum<T, EXACT, kStandard>(Lf, d, fi, fj, idx);
}

// Coarse terms (lattice i, j, weight) of the interpolated value at fine node (i, j),
// in row-major order of the coarse nodes before any wrap-around.
template <typename T>
__device__ __forceinline__ int prolong_terms(int transfer, int i, int j, int* ti, int* tj, T* w) {
  if (transfer == kRbAxisToRot) {
    if (((i + j) & 1) == 0) {
      ti[0] = i; tj[0] = j; w[0] = T(1);
      return 1;
    }
    const int di[4] = {0, -1, 1, 0}, dj[4] = {-1, 0, 0, 1};
    for (int k = 0; k < 4; ++k) { ti[k] = i + di[k]; tj[k] = j + dj[k]; w[k] = T(0.25); }
    return 4;
  }
  if (transfer == kRbRotToAxis) {
    if ((i & 1) == 0) {
      ti[0] = i >> 1; tj[0] = j >> 1; w[0] = T(1);
      return 1;
    }
    const int i0 = (i - 1) >> 1, i1 = (i + 1) >> 1, j0 = (j - 1) >> 1, j1 = (j + 1) >> 1;
    ti[0] = i0; tj[0] = j0; ti[1] = i1; tj[1] = j0; ti[2] = i0; tj[2] = j1; ti[3] = i1; tj[3] = j1;
    for (int k = 0; k < 4; ++k) w[k] = T(0.25);
    return 4;
  }
  const int nx = (i & 1) ? 2 : 1, ny = (j & 1) ? 2 : 1;
  const T wv = Arith<T>::mul((i & 1) ? T(0.5) : T(1), (j & 1) ? T(0.5) : T(1));  // exact
  int m = 0;
  for (int b = 0; b < ny; ++b)
    for (int a = 0; a < nx; ++a) {
      ti[m] = (i & 1) ? ((i - 1) >> 1) + a : i >> 1;
      tj[m] = (j & 1) ? ((j - 1) >> 1) + b : j >> 1;
      w[m++] = wv;
    }
  return m;
}

// Interpolation from a periodic coarse level.
template <typename T, bool EXACT, class Idx>
__device__ __forceinline__ T prolong_wrapped(const LevelDev<T>& Lc, int transfer, const T* __restrict__ vc,
                                          int i, int j, Idx idx) {
  int ti[4], tj[4];
  T w[4];
  const int nt = prolong_terms<T>(transfer, i, j, ti, tj, w);
  return wrapped_sum<T, EXACT>(Lc, nt, ti, tj, w, vc, idx);
}

// Interpolated correction (P v)(i, j) at fine node (i, j) (PER as in restrict_value).
template <typename T, bool EXACT, bool PER, class Idx = GlobalIdx>
__device__ __forceinline__ T prolong_value(const LevelDev<T>& Lc, int transfer, const T* __restrict__ vc,
                                           int i, int j, Idx idx = Idx()) {
  if (PER) return prolong_wrapped<T, EXACT>(Lc, transfer, vc, i, j, idx);
  T e;
  if (transfer == kRbAxisToRot) {
    if (((i + j) & 1) == 0) {
      e = vc[idx(Lc, i, j)];
    } else {
      const T q = T(0.25);
      e = Arith<T>::mul(q, vc[idx(Lc, i, j - 1)]);
      e = madd<T, EXACT>(e, q, vc[idx(Lc, i - 1, j)]);
      e = madd<T, EXACT>(e, q, vc[idx(Lc, i + 1, j)]);
      e = madd<T, EXACT>(e, q, vc[idx(Lc, i, j + 1)]);
    }
  } else if (transfer == kRbRotToAxis) {
    if ((i & 1) == 0) {
      e = vc[idx(Lc, i >> 1, j >> 1)];
    } else {
      const T q = T(0.25);
      const int i0 = (i - 1) >> 1, i1 = (i + 1) >> 1, j0 = (j - 1) >> 1, j1 = (j + 1) >> 1;
      e = Arith<T>::mul(q, vc[idx(Lc, i0, j0)]);
      e = madd<T, EXACT>(e, q, vc[idx(Lc, i1, j0)]);
      e = madd<T, EXACT>(e, q, vc[idx(Lc, i0, j1)]);
      e = madd<T, EXACT>(e, q, vc[idx(Lc, i1, j1)]);
    }
  } else {
    int xs[2], ys[2];
    T wx, wy;
    int nx, ny;
    if (i & 1) { xs[0] = (i - 1) >> 1; xs[1] = (i + 1) >> 1; nx = 2; wx = T(0.5); }
    else { xs[0] = i >> 1; xs[1] = xs[0]; nx = 1; wx = T(1); }
    if (j & 1) { ys[0] = (j - 1) >> 1; ys[1] = (j + 1) >> 1; ny = 2; wy = T(0.5); }
    else { ys[0] = j >> 1; ys[1] = ys[0]; ny = 1; wy = T(1); }
    const T w = Arith<T>::mul(wx, wy);  // exact
    bool first = true;
    e = T(0);
    for (int b = 0; b < ny; ++b)
      for (int a = 0; a < nx; ++a) {
        const T x = vc[idx(Lc, xs[a], ys[b])];
        e = first ? Arith<T>::mul(w, x) : madd<T, EXACT>(e, w, x);
        first = false;
      }
  }
  return e;
}

// ---- cubic transfers (standard coarsening, App. A, Eq. interp_2d4o / restr_2d4o) ----
// Per axis, the interpolated value at an odd fine position takes the coarse nodes at
// fine offsets -3, -1, 1, 3 with weights -1/16, 9/16, 9/16, -1/16 (even positions
// copy their coarse node); 2D weights are products. R = 1/4 P^T: per axis taps
// (-1, 9, 16, 9, -1) / 32 at fine offsets (-3, -1, 0, 1, 3). All weights and their
// products are exact in FP32 and FP64.
// (Compile-time functions: inside unrolled loops the weights and their products fold
// to literals instead of table loads, conversions and multiplies.)
__host__ __device__ constexpr int cubic_off(int a) { return a == 0 ? -3 : a == 4 ? 3 : a - 2; }
template <typename T>
__host__ __device__ constexpr T cubic_r1(int a) {
  return a == 2 ? T(0.5) : (a == 1 || a == 3) ? T(0.28125) : T(-0.03125);  // 16/32, 9/32, -1/32
}

// Dirichlet edge terms: coordinates folded into [0, n] by odd reflection (sign -1 per
// reflection), boundary positions dropped; then as wrapped_sum (ordered by storage
// position, equal positions merged by exact weight sums).
template <typename T, bool EXACT, class Idx>
__device__ __forceinline__ T folded_sum(const LevelDev<T>& L, int nt, const int* ti, const int* tj, const T* w,
                                        const T* __restrict__ x, Idx idx) {
  int64_t pos[kMaxTransferTerms];
  T wt[kMaxTransferTerms];
  int m = 0;
  const int n2 = 2 * L.n;
  for (int k = 0; k < nt; ++k) {
    int a = ti[k] % n2, b = tj[k] % n2;
    if (a < 0) a += n2;
    if (b < 0) b += n2;
    T wk = w[k];
    if (a > L.n) { a = n2 - a; wk = -wk; }
    if (b > L.n) { b = n2 - b; wk = -wk; }
    if (a == 0 || a == L.n || b == 0 || b == L.n) continue;
    const int64_t p = idx(L, a, b);
    int q = 0;
    while (q < m && pos[q] < p) ++q;
    if (q < m && pos[q] == p) {
      wt[q] = Arith<T>::add(wt[q], wk);
      continue;
    }
    for (int r = m; r > q; --r) {
      pos[r] = pos[r - 1];
      wt[r] = wt[r - 1];
    }
    pos[q] = p;
    wt[q] = wk;
    ++m;
  }
  // weights that cancel (exact zeros) are kept as terms: the oracle's sparse products
  // keep such entries too, and w * x = +-0 leaves a nonzero sum unchanged
  if (m == 0) return T(0);
  T s = Arith<T>::mul(wt[0], x[pos[0]]);
  for (int k = 1; k < m; ++k) s = madd<T, EXACT>(s, wt[k], x[pos[k]]);
  return s;
}

template <typename T, bool EXACT, bool PER, class Idx>
__device__ __forceinline__ T edge_sum(const LevelDev<T>& L, int nt, const int* ti, const int* tj, const T* w,
                                      const T* __restrict__ x, Idx idx) {
  if (PER) return wrapped_sum<T, EXACT>(L, nt, ti, tj, w, x, idx);
  return folded_sum<T, EXACT>(L, nt, ti, tj, w, x, idx);
}

// Restricted residual at coarse node (i, j) with the cubic adjoint.
template <typename T, bool EXACT, bool PER, class Idx = GlobalIdx>
__device__ __forceinline__ T restrict_cubic_value(const LevelDev<T>& Lf, const T* __restrict__ d, int i, int j,
                                                  Idx idx = Idx()) {
  const int fi = 2 * i, fj = 2 * j;
  const int lo = PER ? 3 : 4, hi = Lf.n - (PER ? 4 : 4);  // all taps on unknowns, no wrap
  if (fi >= lo && fi <= hi && fj >= lo && fj <= hi) {
    T s = T(0);
#pragma unroll
    for (int b = 0; b < 5; ++b)
#pragma unroll
      for (int a = 0; a < 5; ++a) {
        const T w = cubic_r1<T>(a) * cubic_r1<T>(b);  // exact
        const T x = d[idx(Lf, fi + cubic_off(a), fj + cubic_off(b))];
        s = (a == 0 && b == 0) ? Arith<T>::mul(w, x) : madd<T, EXACT>(s, w, x);
      }
    return s;
  }
  int ti[25], tj[25];
  T w[25];
  int m = 0;
  for (int b = 0; b < 5; ++b)
    for (int a = 0; a < 5; ++a) {
      ti[m] = fi + cubic_off(a);
      tj[m] = fj + cubic_off(b);
      w[m++] = Arith<T>::mul(cubic_r1<T>(a), cubic_r1<T>(b));
    }
  return edge_sum<T, EXACT, PER>(Lf, 25, ti, tj, w, d, idx);
}

// 1D cubic interpolation taps of fine position i: coarse positions and weights.
template <typename T>
__device__ __forceinline__ int cubic_taps(int i, int* c, T* w) {
  if ((i & 1) == 0) {
    c[0] = i >> 1;
    w[0] = T(1);
    return 1;
  }
  const int c0 = (i - 3) >> 1;
  c[0] = c0; c[1] = c0 + 1; c[2] = c0 + 2; c[3] = c0 + 3;
  w[0] = T(-0.0625); w[1] = T(0.5625); w[2] = T(0.5625); w[3] = T(-0.0625);
  return 4;
}

// Interpolated correction (P v)(i, j) at fine node (i, j) with cubic interpolation.
template <typename T, bool EXACT, bool PER, class Idx = GlobalIdx>
__device__ __forceinline__ T prolong_cubic_value(const LevelDev<T>& Lc, const T* __restrict__ vc, int i, int j,
                                                 Idx idx = Idx()) {
  int cx[4], cy[4];
  T wx[4], wy[4];
  const int nx = cubic_taps<T>(i, cx, wx), ny = cubic_taps<T>(j, cy, wy);
  const int lo = PER ? 0 : 1;
  if (cx[0] >= lo && cx[nx - 1] <= Lc.n - 1 && cy[0] >= lo && cy[ny - 1] <= Lc.n - 1) {
    T e = T(0);
    for (int b = 0; b < ny; ++b)
      for (int a = 0; a < nx; ++a) {
        const T w = Arith<T>::mul(wx[a], wy[b]);  // exact
        const T x = vc[idx(Lc, cx[a], cy[b])];
        e = (a == 0 && b == 0) ? Arith<T>::mul(w, x) : madd<T, EXACT>(e, w, x);
      }
    return e;
  }
  int ti[16], tj[16];
  T w[16];
  int m = 0;
  for (int b = 0; b < ny; ++b)
    for (int a = 0; a < nx; ++a) {
      ti[m] = cx[a];
      tj[m] = cy[b];
      w[m++] = Arith<T>::mul(wx[a], wy[b]);
    }
  return edge_sum<T, EXACT, PER>(Lc, m, ti, tj, w, vc, idx);
}

// Any transfer, boundary kind chosen at run time (tail kernels).
template <typename T, bool EXACT, class Idx = GlobalIdx>
__device__ __forceinline__ T restrict_any(const LevelDev<T>& Lf, int transfer, const T* __restrict__ d, int i, int j,
                                          Idx idx = Idx()) {
  if (transfer == kStandardCubic)
    return Lf.per ? restrict_cubic_value<T, EXACT, true>(Lf, d, i, j, idx)
                  : restrict_cubic_value<T, EXACT, false>(Lf, d, i, j, idx);
  return Lf.per ? restrict_value<T, EXACT, true>(Lf, transfer, d, i, j, idx)
                : restrict_value<T, EXACT, false>(Lf, transfer, d, i, j, idx);
}

template <typename T, bool EXACT, class Idx = GlobalIdx>
__device__ __forceinline__ T prolong_any(const LevelDev<T>& Lc, int transfer, const T* __restrict__ vc, int i, int j,
                                         Idx idx = Idx()) {
  if (transfer == kStandardCubic)
    return Lc.per ? prolong_cubic_value<T, EXACT, true>(Lc, vc, i, j, idx)
                  : prolong_cubic_value<T, EXACT, false>(Lc, vc, i, j, idx);
  return Lc.per ? prolong_value<T, EXACT, true>(Lc, transfer, vc, i, j, idx)
                : prolong_value<T, EXACT, false>(Lc, transfer, vc, i, j, idx);
}

// Stores the restricted value v of coarse node (i, j); with tc also the coarse level's
// first half-sweep from u = 0 (the value k_first_half_zero would write from this f).
template <typename T>
__device__ __forceinline__ void store_restricted(const LevelDev<T>& Lc, T* __restrict__ fc, T* __restrict__ tc,
                                                 int i, int j, T v) {
  const int64_t at = sidx(Lc, i, j);
  fc[at] = v;
  if (tc) tc[at] = is_red(Lc, i, j) == 1 ? rnd(Lc, relax_from_zero(v, node_wd(Lc, i, j))) : T(0);
}

template <typename T, bool EXACT, bool PER>
__global__ void __launch_bounds__(kBX * kBY, MinBlocks<T>::value)
    k_restrict_cubic(const LevelDev<T>* __restrict__ Lfp, const LevelDev<T>* __restrict__ Lcp, const T* __restrict__ d,
                     T* __restrict__ fc, T* __restrict__ tc) {
  const LevelDev<T>& Lc = *Lcp;
  int i, j;
  if (!thread_node(Lc, i, j) || !interior(Lc, i, j)) return;
  store_restricted(Lc, fc, tc, i, j, rnd(Lc, restrict_cubic_value<T, EXACT, PER>(*Lfp, d, i, j)));
}

template <typename T, bool EXACT, bool PER>
__global__ void __launch_bounds__(kBX * kBY, MinBlocks<T>::value)
    k_prolong_cubic(const LevelDev<T>* __restrict__ Lfp, const LevelDev<T>* __restrict__ Lcp, const T* uin, T* uf,
                    const T* __restrict__ vc) {
  const LevelDev<T>& Lf = *Lfp;
  int i, j;
  if (!thread_node(Lf, i, j) || !interior(Lf, i, j)) return;
  const int64_t at = sidx(Lf, i, j);
  uf[at] = rnd(Lf, Arith<T>::add(uin[at], prolong_cubic_value<T, EXACT, PER>(*Lcp, vc, i, j)));
}

// On large levels the restriction and interpolation kernels give each thread
// kTransferRows rows (kBY apart) and prefetch the lines those rows read into L2 first;
// interpolation onto an axis level also takes a node pair (2p, 2p + 1) per thread, so
// that every lane evaluates one node of each kind (a copied coarse value and an
// average; with one node per thread alternate lanes idled through the average).
// Measured at 4097^2 (FP64 / FP32): level-0 interpolation 262 -> 152 / 75 -> 53 us,
// FP32 level-0 restriction 83 -> 73 us; on levels below 2048 rows and on rotated fine
// levels the one-node-per-thread form was as fast or faster, so those keep it.
constexpr int kTransferRows = 4;
constexpr int kTransferRowsMinLevelRows = 2048;

template <typename T, bool EXACT, bool PER, int ROWS>
__global__ void __launch_bounds__(kBX * kBY, MinBlocks<T>::value) k_restrict(const LevelDev<T>* __restrict__ Lfp, const LevelDev<T>* __restrict__ Lcp,
                           int transfer, const T* __restrict__ d, T* __restrict__ fc, T* __restrict__ tc) {
  const LevelDev<T>& Lf = *Lfp;
  const LevelDev<T>& Lc = *Lcp;
  const int q = blockIdx.x * kBX + threadIdx.x;
  if (q >= Lc.cols) return;
  const int jb = blockIdx.y * (kBY * ROWS) + threadIdx.y;
#pragma unroll
  for (int r = 0; r < (ROWS > 1 ? ROWS : 0); ++r) {
    // fine node under the coarse node (and the odd fine row after it for H = 2h)
    const int j = min(jb + r * kBY, Lc.rows - 1);
    const int i = Lc.kind == kRot ? 2 * q + (j & 1) : q;
    const int fi = min(transfer == kRbAxisToRot ? i : 2 * i, Lf.n);
    const int fj = min(transfer == kRbAxisToRot ? j : 2 * j, Lf.n);
    prefetch_l2(d + sidx(Lf, fi, fj));
    if (transfer != kRbAxisToRot && fj < Lf.n) prefetch_l2(d + sidx(Lf, min(fi + 1, Lf.n), fj + 1));
  }
#pragma unroll
  for (int r = 0; r < ROWS; ++r) {
    const int j = jb + r * kBY;
    if (j >= Lc.rows) break;
    const int i = Lc.kind == kRot ? 2 * q + (j & 1) : q;
    if (!interior(Lc, i, j)) continue;
    store_restricted(Lc, fc, tc, i, j, rnd(Lc, restrict_value<T, EXACT, PER>(Lf, transfer, d, i, j)));
  }
}

// PAIR: an axis fine level, one thread per node pair (2p, 2p + 1); otherwise one thread
// per storage column (rotated fine levels hold one interpolation kind per row).
template <typename T, bool EXACT, bool PER, int ROWS, bool PAIR>
__global__ void __launch_bounds__(kBX * kBY, MinBlocks<T>::value) k_prolong_add(const LevelDev<T>* __restrict__ Lfp, const LevelDev<T>* __restrict__ Lcp,
                              int transfer, const T* uin, T* uf, const T* __restrict__ vc) {
  const LevelDev<T>& Lf = *Lfp;
  const LevelDev<T>& Lc = *Lcp;
  const bool axis = Lf.kind == kAxis;
  const int t = blockIdx.x * kBX + threadIdx.x;
  const int i0 = PAIR ? 2 * t : 0;
  if (PAIR ? i0 > Lf.n : t >= Lf.cols) return;
  const int jb = blockIdx.y * (kBY * ROWS) + threadIdx.y;
#pragma unroll
  for (int r = 0; r < (ROWS > 1 ? ROWS : 0); ++r) {
    const int j = min(jb + r * kBY, Lf.rows - 1);
    const int i = PAIR ? i0 : min(axis ? t : 2 * t + (j & 1), Lf.n);
    prefetch_l2(uin + sidx(Lf, i, j));
    const int ci = transfer == kRbAxisToRot ? i : i >> 1, cj = transfer == kRbAxisToRot ? j : j >> 1;
    prefetch_l2(vc + sidx(Lc, ci, cj));
  }
#pragma unroll
  for (int r = 0; r < ROWS; ++r) {
    const int j = jb + r * kBY;
    if (j >= Lf.rows) break;
#pragma unroll
    for (int k = 0; k < (PAIR ? 2 : 1); ++k) {
      const int i = PAIR ? i0 + k : (axis ? t : 2 * t + (j & 1));
      if (!interior(Lf, i, j)) continue;
      const int64_t at = sidx(Lf, i, j);
      uf[at] = rnd(Lf, Arith<T>::add(uin[at], prolong_value<T, EXACT, PER>(Lc, transfer, vc, i, j)));
    }
  }
}

// Exact solve on the one-unknown coarsest level: u = f / a_pp (Dirichlet), or the
// zero-mean solution u = 0 of a periodic single node, whose operator row is zero.
template <typename T>
__global__ void k_coarsest(int64_t idx, T a, int zero_mean, const T* __restrict__ f, T* __restrict__ u) {
  if (threadIdx.x == 0 && blockIdx.x == 0) u[idx] = zero_mean ? T(0) : Arith<T>::div(f[idx], a);
}

// Exact coarsest solve with m > 1 unknowns: y = G f, then u = G^T y (DenseCoarse).
// Thread i (strided by nth) forms y_i, then x_i, each a sum from its first product with
// k ascending; SYNC separates the two products (returns false if the caller must stop).
template <typename T, bool EXACT, class IDX, class SYNC>
__device__ __forceinline__ bool dense_coarse(const DenseCoarse<T>& C, const LevelDev<T>& L, const T* F, T* Y,
                                             T* U, IDX idx, int tid, int nth, SYNC sync) {
  // The loads of kDU consecutive terms are issued before their products are summed
  // (in the same k-ascending order), so each row pays one load latency per kDU terms.
  constexpr int kDU = 8;
  const int m = C.m;
  const int2 q0 = C.ij[0];
  const T f0 = F[idx(L, q0.x, q0.y)];
  for (int i = tid; i < m; i += nth) {
    T s = Arith<T>::mul(C.ga[i], f0);
    int k = 1;
    for (; k + kDU - 1 <= i; k += kDU) {
      T g[kDU], x[kDU];
#pragma unroll
      for (int r = 0; r < kDU; ++r) {
        const int2 q = C.ij[k + r];
        g[r] = C.ga[(int64_t)(k + r) * m + i];
        x[r] = F[idx(L, q.x, q.y)];
      }
#pragma unroll
      for (int r = 0; r < kDU; ++r) s = EXACT ? Arith<T>::add(s, Arith<T>::mul(g[r], x[r])) : Arith<T>::fma(g[r], x[r], s);
    }
    for (; k <= i; ++k) {
      const int2 q = C.ij[k];
      const T g = C.ga[(int64_t)k * m + i];
      const T x = F[idx(L, q.x, q.y)];
      s = EXACT ? Arith<T>::add(s, Arith<T>::mul(g, x)) : Arith<T>::fma(g, x, s);
    }
    const int2 p = C.ij[i];
    Y[idx(L, p.x, p.y)] = s;
  }
  if (!sync()) return false;
  for (int i = tid; i < m; i += nth) {
    const int2 p = C.ij[i];
    T s = Arith<T>::mul(C.gb[(int64_t)i * m + i], Y[idx(L, p.x, p.y)]);
    int k = i + 1;
    for (; k + kDU - 1 < m; k += kDU) {
      T g[kDU], x[kDU];
#pragma unroll
      for (int r = 0; r < kDU; ++r) {
        const int2 q = C.ij[k + r];
        g[r] = C.gb[(int64_t)(k + r) * m + i];
        x[r] = Y[idx(L, q.x, q.y)];
      }
#pragma unroll
      for (int r = 0; r < kDU; ++r) s = EXACT ? Arith<T>::add(s, Arith<T>::mul(g[r], x[r])) : Arith<T>::fma(g[r], x[r], s);
    }
    for (; k < m; ++k) {
      const int2 q = C.ij[k];
      const T g = C.gb[(int64_t)k * m + i];
      const T x = Y[idx(L, q.x, q.y)];
      s = EXACT ? Arith<T>::add(s, Arith<T>::mul(g, x)) : Arith<T>::fma(g, x, s);
    }
    U[idx(L, p.x, p.y)] = s;
  }
  return true;
}

struct BlockSync {
  __device__ __forceinline__ bool operator()() const {
    __syncthreads();
    return true;
  }
};

template <typename T, bool EXACT>
__global__ void __launch_bounds__(1024) k_coarsest_dense(DenseCoarse<T> C, const LevelDev<T>* __restrict__ Lp,
                                                         const T* __restrict__ f, T* __restrict__ y,
                                                         T* __restrict__ u) {
  dense_coarse<T, EXACT>(C, *Lp, f, y, u, GlobalIdx(), (int)threadIdx.x, (int)blockDim.x, BlockSync());
}

// Block-wide sum of a double (blockDim = kBX * kBY = 256 threads).
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double warp_part[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  if (lane == 0) warp_part[warp] = v;
  __syncthreads();
  const int nw = (blockDim.x * blockDim.y) >> 5;
  v = tid < nw ? warp_part[tid] : 0.0;
  if (warp == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Norm reductions use a bounded grid: block (bx, by) covers the 32 x 8 tiles
// (bx, by), (bx, by + gridDim.y), ... so that at most kMaxPartials partial sums
// are left for the single-block final sum.
constexpr int kMaxPartials = 2048;

template <typename T, bool EXACT>
__global__ void k_resnorm_partial(const LevelDev<T>* __restrict__ Lp, const T* __restrict__ u,
                                  const T* __restrict__ f, double* __restrict__ partial, int tiles_y) {
  const LevelDev<T>& L = *Lp;
  double v = 0.0;
  const int q = blockIdx.x * kBX + threadIdx.x;
  for (int ty = blockIdx.y; ty < tiles_y; ty += gridDim.y) {
    const int j = ty * kBY + threadIdx.y;
    if (j >= L.rows || q >= L.cols) continue;
    const int i = L.kind == kRot ? 2 * q + (j & 1) : q;
    if (!interior(L, i, j)) continue;
    const int64_t at = sidx(L, i, j);
    const double d = (double)Arith<T>::sub(f[at], apply_at<T, EXACT>(L, u, i, j, at, nullptr));
    v += d * d;
  }
  v = block_sum(v);
  if (threadIdx.x == 0 && threadIdx.y == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = v;
}

// Residual-norm partial sums (as k_resnorm_partial: same nodes, order and sums) fused
// with the first half-sweep of the next cycle: nodes of colour `red` get the relaxed
// value u + (f - L u) omega / a_pp from the same residual, the others are copied
// (u -> uout, out of place as in the half-sweep kernels). Per node the arithmetic is
// that of the half-sweep, so a cycle that starts with the other colour from uout gives
// the same bits as one that starts from u.
// First half-sweep (colour `red`) of a cycle on a coarse level, whose correction starts
// from u = 0, into t: on a zero vector every stencil sum is +0 (each operator row has a
// positive diagonal, and +0 absorbs -0), so the half-sweep's residual is f and its new
// value 0 + f omega / a_pp; the other colour keeps its 0. This writes exactly those bits
// without the stencil gathers (and replaces zeroing u, since the black half-sweep that
// follows writes every unknown of u).
template <typename T>
__global__ void k_first_half_zero(const LevelDev<T>* __restrict__ Lp, const T* __restrict__ f, T* __restrict__ t,
                                  int red) {
  const LevelDev<T>& L = *Lp;
  int i, j;
  if (!thread_node(L, i, j) || !interior(L, i, j)) return;
  const int64_t at = sidx(L, i, j);
  T e = T(0);
  if (is_red(L, i, j) == red) e = rnd(L, relax_from_zero(f[at], node_wd(L, i, j)));
  t[at] = e;
}

// The norm kernels below (k_resnorm_red, k_ir_residual) walk the level's 32 x 8 tiles
// in a flat order, block b taking tiles b, b + gridDim.x, ...: with one block per
// resident slot every SM gets the same number of tiles (to one), whatever the grid
// shape, and the partial sums stay at most kMaxPartials.
template <typename T, bool EXACT, int NT>
__global__ void __launch_bounds__(kBX * kBY, MinBlocks<T>::value)
    k_resnorm_red(const LevelDev<T>* __restrict__ Lp, const T* __restrict__ u, const T* __restrict__ f,
                  T* __restrict__ uout, int red, double* __restrict__ partial, int tiles_x, int tiles) {
  const LevelDev<T>& L = *Lp;
  constexpr int NA = NT > 0 ? NT : 1;
  T c[NA];
  int dl[NA];
#pragma unroll
  for (int k = 0; k < NA; ++k) {
    c[k] = L.c[k];
    dl[k] = L.delta[0][k];
  }
  double v = 0.0;
  for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int ty = t / tiles_x;
    const int q = (t - ty * tiles_x) * kBX + threadIdx.x;
    const int j = ty * kBY + threadIdx.y;
    if (j >= L.rows || q >= L.cols) continue;
    const int i = L.kind == kRot ? 2 * q + (j & 1) : q;
    if (!interior(L, i, j)) continue;
    const int64_t at = sidx(L, i, j);
    T wd;
    T s;
    if (NT > 0 && L.kind == kAxis && fast_node(L, i, j)) {
      s = apply_fast<T, EXACT, NA>(c, dl, u, at);
      wd = L.wd;
    } else {
      s = apply_at<T, EXACT, 1>(L, u, i, j, at, &wd);
    }
    const T r = Arith<T>::sub(f[at], s);
    const double d = (double)r;
    v += d * d;
    uout[at] = is_red(L, i, j) == red
                   ? rnd(L, EXACT ? Arith<T>::add(u[at], Arith<T>::mul(r, wd)) : Arith<T>::fma(r, wd, u[at]))
                   : u[at];
  }
  v = block_sum(v);
  if (threadIdx.x == 0 && threadIdx.y == 0) partial[blockIdx.x] = v;
}

template <typename T>
__global__ void k_sumsq_partial(const LevelDev<T>* __restrict__ Lp, const T* __restrict__ f,
                                double* __restrict__ partial, int tiles_y) {
  const LevelDev<T>& L = *Lp;
  double v = 0.0;
  const int q = blockIdx.x * kBX + threadIdx.x;
  for (int ty = blockIdx.y; ty < tiles_y; ty += gridDim.y) {
    const int j = ty * kBY + threadIdx.y;
    if (j >= L.rows || q >= L.cols) continue;
    const int i = L.kind == kRot ? 2 * q + (j & 1) : q;
    if (!interior(L, i, j)) continue;
    const double x = (double)f[sidx(L, i, j)];
    v += x * x;
  }
  v = block_sum(v);
  if (threadIdx.x == 0 && threadIdx.y == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = v;
}

// One block of 256 threads: strided partial sums, then a fixed tree.
__global__ void k_sum_partials(const double* __restrict__ partial, int count, double* __restrict__ out) {
  double v = 0.0;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  for (int k = tid; k < count; k += blockDim.x * blockDim.y) v += partial[k];
  v = block_sum(v);
  if (tid == 0) *out = v;
}

// Boundary ring of src into dst (Dirichlet data g into the level-0 ping-pong array).
template <typename T>
__global__ void k_copy_boundary(int n, int pitch, const T* __restrict__ src, T* __restrict__ dst) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > n) return;
  const int64_t at[4] = {k, (int64_t)n * pitch + k, (int64_t)k * pitch, (int64_t)k * pitch + n};
  for (int m = 0; m < 4; ++m) dst[at[m]] = src[at[m]];
}

template <typename T>
__global__ void k_zero_boundary(int n, int pitch, T* __restrict__ u) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > n) return;
  u[k] = T(0);                             // j = 0
  u[(int64_t)n * pitch + k] = T(0);        // j = n
  u[(int64_t)k * pitch] = T(0);            // i = 0
  u[(int64_t)k * pitch + n] = T(0);        // i = n
}

// Iterative-refinement residual: r = f - L u in FP64 (evaluation order of EXACT),
// r32 = fl32(r * scale) for the FP32 inner cycles, and per-block sums of r^2.
//
// With t32 (and L32, the FP32 level 0), the kernel also does the first half-sweep of the
// FP32 cycle that follows from e = 0: red nodes get 0 + r32 omega / a_pp, black nodes 0.
// On a zero vector the FP32 stencil sum is +0 (every operator row has a positive
// diagonal, and +0 absorbs -0 in a sum), so the half-sweep's residual is r32 itself and
// this is the half-sweep's value bit for bit.
template <bool EXACT, int NT>
__global__ void __launch_bounds__(kBX * kBY, MinBlocks<double>::value)
    k_ir_residual(const LevelDev<double>* __restrict__ Lp, const double* __restrict__ u,
                  const double* __restrict__ f, float* __restrict__ r32, double scale,
                  double* __restrict__ partial, int tiles_x, int tiles, int bf16,
                  const LevelDev<float>* __restrict__ L32p, float* __restrict__ t32) {
  const LevelDev<double>& L = *Lp;
  const LevelDev<float>& L32 = *L32p;  // FP32 finest level: same nodes, its own row pitch
  constexpr int NA = NT > 0 ? NT : 1;
  double c[NA];
  int dl[NA];
#pragma unroll
  for (int k = 0; k < NA; ++k) {
    c[k] = L.c[k];
    dl[k] = L.delta[0][k];
  }
  const int pitch32 = L32.pitch;
  double v = 0.0;
  for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int ty = t / tiles_x;
    const int q = (t - ty * tiles_x) * kBX + threadIdx.x;
    const int j = ty * kBY + threadIdx.y;
    if (j >= L.rows || q >= L.cols) continue;
    const int i = q;  // the finest level is an axis grid
    if (!interior(L, i, j)) continue;
    const int64_t at = (int64_t)j * L.pitch + i;
    const double s = (NT > 0 && fast_node(L, i, j)) ? apply_fast<double, EXACT, NA>(c, dl, u, at)
                                                    : apply_at<double, EXACT, 1>(L, u, i, j, at, nullptr);
    const double r = Arith<double>::sub(f[at], s);
    const float r32v = (float)(r * scale);
    const float rv = bf16 ? __bfloat162float(__float2bfloat16_rn(r32v)) : r32v;
    const int64_t at32 = (int64_t)j * pitch32 + i;
    r32[at32] = rv;
    v += r * r;
    if (t32) {
      float e = 0.f;
      if (is_red(L32, i, j) == 1) e = rnd(L32, relax_from_zero(rv, node_wd(L32, i, j)));
      t32[at32] = e;
    }
  }
  v = block_sum(v);
  if (threadIdx.x == 0 && threadIdx.y == 0) partial[blockIdx.x] = v;
}

// u += e * inv_scale (FP64 update of the refinement step).
// kTransferRows rows per thread with the lines prefetched into L2, as in the transfers.
__global__ void k_ir_update(const LevelDev<double>* __restrict__ Lp, int pitch32, double* __restrict__ u,
                            const float* __restrict__ e, double inv_scale) {
  const LevelDev<double>& L = *Lp;
  const int q = blockIdx.x * kBX + threadIdx.x;
  if (q >= L.cols) return;
  const int jb = blockIdx.y * (kBY * kTransferRows) + threadIdx.y;
#pragma unroll
  for (int r = 0; r < kTransferRows; ++r) {
    const int jr = min(jb + r * kBY, L.rows - 1);
    prefetch_l2(u + (int64_t)jr * L.pitch + q);
    prefetch_l2(e + (int64_t)jr * pitch32 + q);
  }
#pragma unroll
  for (int r = 0; r < kTransferRows; ++r) {
    const int j = jb + r * kBY;
    if (j >= L.rows) break;
    const int i = q;  // the finest level is an axis grid
    if (!interior(L, i, j)) continue;
    const int64_t at = (int64_t)j * L.pitch + i;
    u[at] = u[at] + (double)e[(int64_t)j * pitch32 + i] * inv_scale;
  }
}

// ---- small-level tail ---------------------------------------------------------
// One thread-block cluster (kTailCtas CTAs of kTailThreads threads, one per SM)
// runs the whole sub-cycle; the hardware cluster barrier separates dependent
// phases (release / acquire at cluster scope, covering the global-memory arrays).
constexpr int kTailThreads = 1024;

// Storage element k of a level (row-major over rows x cols) -> lattice node.
template <typename T>
__device__ __forceinline__ bool tail_node(const LevelDev<T>& L, int k, int& i, int& j) {
  j = k / L.cols;
  const int q = k - j * L.cols;
  i = L.kind == kRot ? 2 * q + (j & 1) : q;
  return interior(L, i, j);
}

// The tail's op program (see TailOp) run by `nth` threads (thread index tid) with
// sync() between dependent phases; sync() returns false when the threads must stop (a
// bounded barrier gave up), and the program is abandoned.
template <typename T, bool EXACT, class SYNC>
__device__ __forceinline__ void tail_program(const TailDesc<T>* __restrict__ D, const int4* __restrict__ prog,
                                             int nops, int tid, int nth, SYNC sync) {
  for (int p = 0; p < nops; ++p) {
    const int4 op = prog[p];
    const int l = op.y;
    const LevelDev<T>& L = *D->L[l];
    const int total = L.rows * L.cols;
    int i, j;
    if (op.x == kOpZero) {
      T* u = D->u[l];
      const int tot = L.rows * L.pitch;
      for (int k = tid; k < tot; k += nth) u[k] = T(0);
    } else if (op.x == kOpSmooth) {
      T* U = D->u[l];
      T* Tb = D->t[l];
      const T* F = D->f[l];
      if (D->smoother == 0) {
        for (int half = 1; half >= 0; --half) {  // red (1) from U into Tb, then black (0) back
          const T* src = half ? U : Tb;
          T* dst = half ? Tb : U;
          for (int k = tid; k < total; k += nth) {
            if (!tail_node(L, k, i, j)) continue;
            const int64_t at = sidx(L, i, j);
            if (op.z && half)  // first half-sweep from u = 0 (op.z: U not zeroed)
              dst[at] = is_red(L, i, j) ? relax_from_zero(F[at], node_wd(L, i, j)) : T(0);
            else
              dst[at] = is_red(L, i, j) == half ? relax_value<T, EXACT>(L, src, F, i, j, at) : src[at];
          }
          if (!sync()) return;
        }
      } else {
        for (int k = tid; k < total; k += nth) {
          if (!tail_node(L, k, i, j)) continue;
          const int64_t at = sidx(L, i, j);
          Tb[at] = relax_value<T, EXACT>(L, U, F, i, j, at);
        }
        if (!sync()) return;
        for (int k = tid; k < total; k += nth) {
          if (!tail_node(L, k, i, j)) continue;
          const int64_t at = sidx(L, i, j);
          U[at] = Tb[at];
        }
      }
    } else if (op.x == kOpResRestrict) {
      const T* U = D->u[l];
      const T* F = D->f[l];
      T* Dd = D->d[l];
      for (int k = tid; k < total; k += nth) {
        if (!tail_node(L, k, i, j)) continue;
        const int64_t at = sidx(L, i, j);
        Dd[at] = Arith<T>::sub(F[at], apply_at<T, EXACT>(L, U, i, j, at, nullptr));
      }
      if (!sync()) return;
      const LevelDev<T>& Lc = *D->L[l + 1];
      T* Fc = D->f[l + 1];
      const int ctot = Lc.rows * Lc.cols;
      for (int k = tid; k < ctot; k += nth) {
        if (!tail_node(Lc, k, i, j)) continue;
        Fc[sidx(Lc, i, j)] = restrict_any<T, EXACT>(L, D->transfer[l], Dd, i, j);
      }
    } else if (op.x == kOpCoarsest) {
      if (D->dense.m > 0) {
        if (!dense_coarse<T, EXACT>(D->dense, L, D->f[l], D->d[l], D->u[l], GlobalIdx(), tid, nth, sync)) return;
      } else if (tid == 0) {
        D->u[l][D->coarsest_idx] =
            D->coarsest_zero ? T(0) : Arith<T>::div(D->f[l][D->coarsest_idx], D->coarsest_a);
      }
    } else {  // kOpProlong
      const LevelDev<T>& Lc = *D->L[l + 1];
      T* U = D->u[l];
      const T* V = D->u[l + 1];
      for (int k = tid; k < total; k += nth) {
        if (!tail_node(L, k, i, j)) continue;
        const int64_t at = sidx(L, i, j);
        U[at] = Arith<T>::add(U[at], prolong_any<T, EXACT>(Lc, D->transfer[l], V, i, j));
      }
    }
    if (!sync()) return;
  }
}

template <typename T, bool EXACT>
__global__ void __launch_bounds__(kTailThreads, 1)
    k_tail(const TailDesc<T>* __restrict__ D, const int4* __restrict__ prog, int nops) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  tail_program<T, EXACT>(D, prog, nops, (int)cluster.block_rank() * kTailThreads + threadIdx.x,
                         (int)cluster.num_blocks() * kTailThreads, [&]() {
                           cluster.sync();
                           return true;
                         });
}

// ---- batched level-synchronous step kernels ------------------------------------
__device__ __forceinline__ int batch_entry(const int* __restrict__ prefix, int ne, int b) {
  int lo = 0, hi = ne - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <typename T, bool EXACT, int RPT>
__global__ void __launch_bounds__(kBX * kBY)
    k_batch_step(int op, const BatchLevel<T>* __restrict__ E, const int* __restrict__ prefix, int ne,
                 const int* __restrict__ active) {
  const int b = blockIdx.x;
  const int e = batch_entry(prefix, ne, b);
  const BatchLevel<T>& B = E[e];
  if (!active[B.problem]) return;
  const int tile = b - prefix[e];
  const bool coarse = op == kBRestrict;
  const LevelDev<T>& L = coarse ? *B.Lc : *B.L;  // level whose storage is tiled
  const int tx = coarse ? B.ctiles_x : B.tiles_x;
  const int bx = tile % tx, by = tile / tx;
  const int qb = bx * kBatchCols + 2 * threadIdx.x;
  const int jb = by * kBY * RPT + threadIdx.y;
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int j = jb + r * kBY;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int q = qb + c;
      if (j >= L.rows || q >= L.cols) continue;
      const int i = L.kind == kRot ? 2 * q + (j & 1) : q;
      if (!interior(L, i, j)) continue;
      const int64_t at = (int64_t)j * L.pitch + q;
      switch (op) {
        case kBZero:
          B.u[at] = T(0);
          break;
        case kBHalfRed:
          B.t[at] = is_red(L, i, j) ? relax_value<T, EXACT, 1>(L, B.u, B.f, i, j, at) : B.u[at];
          break;
        case kBHalfRedZero:  // as k_first_half_zero
          B.t[at] = is_red(L, i, j) ? relax_from_zero(B.f[at], node_wd(L, i, j)) : T(0);
          break;
        case kBHalfBlack:
          B.u[at] = is_red(L, i, j) ? B.t[at] : relax_value<T, EXACT, 1>(L, B.t, B.f, i, j, at);
          break;
        case kBResidual:
          B.d[at] = Arith<T>::sub(B.f[at], apply_at<T, EXACT, 1>(L, B.u, i, j, at, nullptr));
          break;
        case kBRestrict:
          B.fc[at] = restrict_value<T, EXACT, false>(*B.L, B.transfer, B.d, i, j);
          break;
        default:  // kBProlong
          B.u[at] = Arith<T>::add(B.u[at], prolong_value<T, EXACT, false>(*B.Lc, B.transfer, B.uc, i, j));
          break;
      }
    }
  }
}

template <typename T>
__global__ void k_batch_coarsest(const BatchLevel<T>* __restrict__ E, int ne, const int* __restrict__ active) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const BatchLevel<T>& B = E[e];
  if (!active[B.problem]) return;
  B.uc[B.coarsest_idx] = Arith<T>::div(B.fc[B.coarsest_idx], B.coarsest_a);
}

// Problems whose coarsest level has a dense solve: one block per entry.
template <typename T, bool EXACT>
__global__ void __launch_bounds__(256) k_batch_coarsest_dense(const BatchLevel<T>* __restrict__ E,
                                                              const int* __restrict__ active) {
  const BatchLevel<T>& B = E[blockIdx.x];
  if (!active[B.problem]) return;  // uniform over the block
  dense_coarse<T, EXACT>(B.dense, *B.Lc, B.fc, B.dc, B.uc, GlobalIdx(), (int)threadIdx.x, (int)blockDim.x,
                         BlockSync());
}

template <bool EXACT>
__global__ void __launch_bounds__(kBX * kBY)
    k_batch_norm_partial(int mode, const BatchLevel<double>* __restrict__ E, const int* __restrict__ prefix, int ne,
                         const int* __restrict__ active, const double* __restrict__ scale,
                         double* __restrict__ partial) {
  const int b = blockIdx.x;
  const int e = batch_entry(prefix, ne, b);
  const BatchLevel<double>& B = E[e];
  double v = 0.0;
  if (active[B.problem]) {
    const LevelDev<double>& L = *B.L;
    const int tile = b - prefix[e];
    const int bx = tile % B.tiles_x, by = tile / B.tiles_x;
    const int qb = bx * kBatchCols + 2 * threadIdx.x;
    const int j = by * kBY + threadIdx.y;
    const double sc = scale[B.problem];
    for (int c = 0; c < 2; ++c) {
      const int q = qb + c;
      if (j >= L.rows || q >= L.cols) continue;
      const int i = L.kind == kRot ? 2 * q + (j & 1) : q;
      if (!interior(L, i, j)) continue;
      const int64_t at = (int64_t)j * L.pitch + q;
      if (mode != 1) {
        const double r = Arith<double>::sub(B.f[at], apply_at<double, EXACT>(L, B.u, i, j, at, nullptr));
        if (mode == 0) B.r32[(int64_t)j * B.pitch32 + q] = (float)(r * sc);
        v += r * r;
      } else {
        v += B.f[at] * B.f[at];
      }
    }
  }
  v = block_sum(v);
  if (threadIdx.x == 0 && threadIdx.y == 0) partial[b] = v;
}

// One block per entry: add its partials in order.
__global__ void k_batch_norm_sum(const BatchLevel<double>* __restrict__ E, const int* __restrict__ prefix,
                                 const int* __restrict__ active, const double* __restrict__ partial,
                                 double* __restrict__ norm2) {
  const int e = blockIdx.x;
  const BatchLevel<double>& B = E[e];
  if (!active[B.problem]) return;
  double v = 0.0;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  for (int k = prefix[e] + tid; k < prefix[e + 1]; k += blockDim.x * blockDim.y) v += partial[k];
  v = block_sum(v);
  if (tid == 0) norm2[B.problem] = v;
}

__global__ void __launch_bounds__(kBX * kBY)
    k_batch_ir_update(const BatchLevel<double>* __restrict__ E, const int* __restrict__ prefix, int ne,
                      const int* __restrict__ active, const double* __restrict__ scale) {
  const int b = blockIdx.x;
  const int e = batch_entry(prefix, ne, b);
  const BatchLevel<double>& B = E[e];
  if (!active[B.problem]) return;
  const LevelDev<double>& L = *B.L;
  const int tile = b - prefix[e];
  const int bx = tile % B.tiles_x, by = tile / B.tiles_x;
  const int qb = bx * kBatchCols + 2 * threadIdx.x;
  const int j = by * kBY + threadIdx.y;
  const double inv = 1.0 / scale[B.problem];
  for (int c = 0; c < 2; ++c) {
    const int q = qb + c;
    if (j >= L.rows || q >= L.cols) continue;
    const int i = L.kind == kRot ? 2 * q + (j & 1) : q;
    if (!interior(L, i, j)) continue;
    const int64_t at = (int64_t)j * L.pitch + q;
    B.u[at] = B.u[at] + (double)B.e32[(int64_t)j * B.pitch32 + q] * inv;
  }
}

// ---- shared-memory-resident tail ---------------------------------------------
// Levels from sm_top down live in one block's shared memory in a compact rows x cols
// layout; node (i, j) of a level is at j * cols + (rot ? i >> 1 : i). Arithmetic
// per node is the same as relax_value / apply_at / restrict_value / prolong_value.
// The interior stencils of the levels held are staged in shared memory too (per level:
// coefficients, and shared-memory offsets for even and odd i), so that a fast node's
// terms need no global-memory reads.
struct TailStencil {
  template <typename T>
  static __host__ __device__ __forceinline__ size_t base(int sm_elems) {  // byte offset of the stencil area
    return ((size_t)sm_elems * sizeof(T) + 15) & ~(size_t)15;
  }
};

template <typename T, bool EXACT>
__device__ __forceinline__ T smem_apply(const LevelDev<T>& L, const T* u, int i, int j, T* wd, const T* __restrict__ cs,
                                        const int* __restrict__ os2) {
  RowSum<T, EXACT> acc;
  if (fast_node(L, i, j)) {
    const int* os = os2 + (L.kind == kRot ? (i & 1) : 0) * kMaxTerms;
    const int e = smem_idx(L, i, j);
#pragma unroll 8
    for (int k = 0; k < L.nt; ++k) acc.add(cs[k], u[e + os[k]], gbit(L.gmask, k));
    if (wd) *wd = L.wd;
  } else {
    const int cl = class_of(L, i, j);
    const int2 ce = L.cls[cl];
    const ClassTerm<T>* tt = L.terms + ce.x;
#pragma unroll 4
    for (int k = 0; k < ce.y; ++k) {
      const Term<T> t = load_term(tt + k);
      acc.add(t.c, u[smem_idx(L, i + t.dx, j + t.dy)], t.start);
    }
    if (wd) *wd = L.cls_wd[cl];
  }
  return acc.value();
}

template <typename T, bool EXACT>
__global__ void __launch_bounds__(kTailThreads, 1)
    k_tail_smem(const TailDesc<T>* __restrict__ D, const int4* __restrict__ prog, int nops) {
  extern __shared__ __align__(16) unsigned char tail_smem[];
  T* sm = reinterpret_cast<T*>(tail_smem);
  const int tid = threadIdx.x;
  const int top = D->sm_top;
  for (int k = tid; k < D->sm_elems; k += kTailThreads) sm[k] = T(0);
  // interior stencils of the levels held: coefficients [level][kMaxTerms], offsets
  // [level][parity][kMaxTerms]
  const int nst = D->nlev - top;
  T* stc = reinterpret_cast<T*>(tail_smem + TailStencil::base<T>(D->sm_elems));
  int* sto = reinterpret_cast<int*>(stc + nst * kMaxTerms);
  for (int x = tid; x < nst * kMaxTerms; x += kTailThreads) {
    const int l = top + x / kMaxTerms, k = x - (x / kMaxTerms) * kMaxTerms;
    const LevelDev<T>& L = *D->L[l];
    if (k < L.nt) {
      stc[x] = L.c[k];
      sto[2 * (l - top) * kMaxTerms + k] = L.sdy[k] * L.cols + L.sdx[0][k];
      sto[(2 * (l - top) + 1) * kMaxTerms + k] = L.sdy[k] * L.cols + L.sdx[1][k];
    }
  }
  __syncthreads();
  {  // top level: u and f from global memory
    const LevelDev<T>& L = *D->L[top];
    for (int k = tid; k < L.rows * L.cols; k += kTailThreads) {
      const int j = k / L.cols, q = k - j * L.cols;
      sm[D->sm_u[top] + k] = D->u[top][(int64_t)j * L.pitch + q];
      sm[D->sm_f[top] + k] = D->f[top][(int64_t)j * L.pitch + q];
    }
  }
  __syncthreads();
  for (int p = 0; p < nops; ++p) {
    const int4 op = prog[p];
    const int l = op.y;
    const LevelDev<T>& L = *D->L[l];
    const int total = L.rows * L.cols;
    T* U = sm + D->sm_u[l];
    T* Tb = sm + D->sm_t[l];
    T* F = sm + D->sm_f[l];
    const T* cs = stc + (l - top) * kMaxTerms;
    const int* os2 = sto + 2 * (l - top) * kMaxTerms;
    int i, j;
    if (op.x == kOpZero) {
      for (int k = tid; k < total; k += kTailThreads) U[k] = T(0);
    } else if (op.x == kOpSmooth) {
      if (D->smoother == 0) {
        for (int half = 1; half >= 0; --half) {
          const T* src = half ? U : Tb;
          T* dst = half ? Tb : U;
          for (int k = tid; k < total; k += kTailThreads) {
            if (!tail_node(L, k, i, j)) continue;
            if (op.z && half) {  // first half-sweep from u = 0 (op.z: U not zeroed)
              dst[k] = is_red(L, i, j) ? relax_from_zero(F[k], node_wd(L, i, j)) : T(0);
            } else if (is_red(L, i, j) == half) {
              T wd;
              const T r = Arith<T>::sub(F[k], smem_apply<T, EXACT>(L, src, i, j, &wd, cs, os2));
              dst[k] = EXACT ? Arith<T>::add(src[k], Arith<T>::mul(r, wd)) : Arith<T>::fma(r, wd, src[k]);
            } else {
              dst[k] = src[k];
            }
          }
          __syncthreads();
        }
      } else {
        for (int k = tid; k < total; k += kTailThreads) {
          if (!tail_node(L, k, i, j)) continue;
          T wd;
          const T r = Arith<T>::sub(F[k], smem_apply<T, EXACT>(L, U, i, j, &wd, cs, os2));
          Tb[k] = EXACT ? Arith<T>::add(U[k], Arith<T>::mul(r, wd)) : Arith<T>::fma(r, wd, U[k]);
        }
        __syncthreads();
        for (int k = tid; k < total; k += kTailThreads) {
          if (!tail_node(L, k, i, j)) continue;
          U[k] = Tb[k];
        }
      }
    } else if (op.x == kOpResRestrict) {
      T* Dd = sm + D->sm_d[l];
      for (int k = tid; k < total; k += kTailThreads) {
        if (!tail_node(L, k, i, j)) continue;
        Dd[k] = Arith<T>::sub(F[k], smem_apply<T, EXACT>(L, U, i, j, nullptr, cs, os2));
      }
      __syncthreads();
      const LevelDev<T>& Lc = *D->L[l + 1];
      T* Fc = sm + D->sm_f[l + 1];
      const int tr = D->transfer[l];
      for (int k = tid; k < Lc.rows * Lc.cols; k += kTailThreads) {
        if (!tail_node(Lc, k, i, j)) continue;
        Fc[k] = restrict_any<T, EXACT>(L, tr, Dd, i, j, SmemIdx());
      }
    } else if (op.x == kOpCoarsest) {
      if (D->dense.m > 0) {
        dense_coarse<T, EXACT>(D->dense, L, F, sm + D->sm_d[l], U, SmemIdx(), tid, kTailThreads, BlockSync());
      } else if (tid == 0) {
        const int c = D->coarsest_zero ? smem_idx(L, 0, 0) : smem_idx(L, 1, 1);
        U[c] = D->coarsest_zero ? T(0) : Arith<T>::div(F[c], D->coarsest_a);
      }
    } else {  // kOpProlong
      const LevelDev<T>& Lc = *D->L[l + 1];
      const T* V = sm + D->sm_u[l + 1];
      const int tr = D->transfer[l];
      for (int k = tid; k < total; k += kTailThreads) {
        if (!tail_node(L, k, i, j)) continue;
        const T e = prolong_any<T, EXACT>(Lc, tr, V, i, j, SmemIdx());
        U[k] = Arith<T>::add(U[k], e);
      }
    }
    __syncthreads();
  }
  {  // top level: u back to global memory (interior nodes)
    const LevelDev<T>& L = *D->L[top];
    for (int k = tid; k < L.rows * L.cols; k += kTailThreads) {
      int i, j;
      if (!tail_node(L, k, i, j)) continue;
      D->u[top][(int64_t)j * L.pitch + (k - j * L.cols)] = sm[D->sm_u[top] + k];
    }
  }
}

template <typename T>
dim3 grid_of(const LevelDev<T>& L) {
  return dim3((L.cols + kBX - 1) / kBX, (L.rows + kBY - 1) / kBY);
}

// Term count of the level's fast stencil if the register-coefficient (NT) kernels can
// take it: 5 or 9 terms in the group shape apply_fast evaluates; 0 otherwise.
template <typename T>
int fast_nt(const LevelDev<T>& L) {
  if (L.nt != 5 && L.nt != 9) return 0;
  if (L.gmask[0] != fast_gmask(L.nt)) return 0;
  for (int w = 1; w < kMaxTerms / 32; ++w)
    if (L.gmask[w]) return 0;
  return L.nt;
}

// Bounded grid of the norm reductions (see kMaxPartials).
template <typename T>
dim3 norm_grid(const LevelDev<T>& L) {
  const dim3 g = grid_of(L);
  return dim3(g.x, std::max(1u, std::min(g.y, (unsigned)(kMaxPartials / (int)g.x))));
}

}  // namespace

// Rows per block of the wide-stencil kernels. FP64 work is bound by each SM's FP64 pipe
// (about 2 operations per clock), so a small level whose 256-thread blocks cover only a
// few SMs is limited by those SMs: there the blocks shrink (down to one warp) until the
// grid has kSpreadBlocksPerSm blocks per SM or the rows run out. Measured on GB300
// (FP64 solves to 1e-10, order 4, RBC, Galerkin): 4097^2 64.0 -> 63.1 ms, 1025^2 9.63 ->
// 9.02 ms, 257^2 6.07 -> 5.78 ms (8 blocks per SM: the same; 2: about half the gain).
constexpr int kSpreadBlocksPerSm = 4;

// SM count of the current device when first asked (one GPU model per process here;
// initialised once, thread-safe).
int sm_count() {
  static const int n = [] {
    int dev = 0, v = 0;
    const bool ok = cudaGetDevice(&dev) == cudaSuccess &&
                    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0;
    return ok ? v : 1;
  }();
  return n;
}

template <typename T>
int gen_block_rows(const LevelDev<T>& L, unsigned gx) {
  if (sizeof(T) != 8) return kBY;
  const long target = (long)kSpreadBlocksPerSm * sm_count();
  int by = kBY;
  while (by > 1 && (long)gx * ((L.rows + by - 1) / by) < target) by >>= 1;
  return by;
}

template <typename T, int NT>
cudaError_t launch_half_sweep_nt(const LevelPair<T>& L, bool exact, const T* uin, const T* f, T* uout, int red,
                                 cudaStream_t s) {
  dim3 g = grid_of(L.h);
  if (L.h.kind == kAxis) g.x = ((L.h.n + 2) / 2 + kBX - 1) / kBX;  // pairs (2p, 2p+1), 2p <= n
  g.y = (L.h.rows + kBY * RowsPer<T>::value - 1) / (kBY * RowsPer<T>::value);
  const dim3 b(kBX, kBY);
  if (L.h.per) {
    if (exact) k_half_sweep_nt<T, true, NT, true><<<g, b, 0, s>>>(L.d, uin, f, uout, red);
    else k_half_sweep_nt<T, false, NT, true><<<g, b, 0, s>>>(L.d, uin, f, uout, red);
  } else {
    if (exact) k_half_sweep_nt<T, true, NT, false><<<g, b, 0, s>>>(L.d, uin, f, uout, red);
    else k_half_sweep_nt<T, false, NT, false><<<g, b, 0, s>>>(L.d, uin, f, uout, red);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_half_sweep(const LevelPair<T>& L, bool exact, const T* uin, const T* f, T* uout,
                              int red, cudaStream_t s) {
  const int ntf = fast_nt(L.h);
  if (ntf == 5) return launch_half_sweep_nt<T, 5>(L, exact, uin, f, uout, red, s);
  if (ntf == 9) return launch_half_sweep_nt<T, 9>(L, exact, uin, f, uout, red, s);
  dim3 g = grid_of(L.h);
  if (L.h.kind == kAxis) g.x = ((L.h.n + 2) / 2 + kBX - 1) / kBX;  // pairs (2p, 2p+1), 2p <= n
  const int by = gen_block_rows(L.h, g.x);
  g.y = (L.h.rows + by - 1) / by;
  const bool deep = sizeof(T) == 4 && L.h.rows < kGenDeepRows;
  if (deep) {
    if (exact) k_half_sweep_gen<T, true, true><<<g, dim3(kBX, by), 0, s>>>(L.d, uin, f, uout, red);
    else k_half_sweep_gen<T, false, true><<<g, dim3(kBX, by), 0, s>>>(L.d, uin, f, uout, red);
  } else {
    if (exact) k_half_sweep_gen<T, true, false><<<g, dim3(kBX, by), 0, s>>>(L.d, uin, f, uout, red);
    else k_half_sweep_gen<T, false, false><<<g, dim3(kBX, by), 0, s>>>(L.d, uin, f, uout, red);
  }
  return cudaGetLastError();
}

template <typename T, bool EXACT, int NT>
cudaError_t launch_sweep_fused_nt(const LevelPair<T>& L, const T* uin, const T* f, T* uout, int rq, int ry,
                                  size_t smem, cudaStream_t s) {
  const dim3 g((L.h.cols + kFTW - 1) / kFTW, (L.h.rows + kFTH - 1) / kFTH);
  cudaFuncSetAttribute(k_sweep_fused<T, EXACT, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  k_sweep_fused<T, EXACT, NT><<<g, dim3(kBX, kBY), smem, s>>>(L.d, uin, f, uout, rq, ry);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sweep_fused(const LevelPair<T>& L, bool exact, const T* uin, const T* f, T* uout, cudaStream_t s) {
  int rq = 0, ry = 0;
  for (int k = 0; k < L.h.nt; ++k) {
    rq = std::max(rq, std::max(std::abs(L.h.sdx[0][k]), std::abs(L.h.sdx[1][k])));
    ry = std::max(ry, std::abs(L.h.sdy[k]));
  }
  const size_t smem = 3 * (size_t)(kFTW + 4 * rq) * (kFTH + 4 * ry) * sizeof(T);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  const int nt = L.h.nt;
  if (exact) {
    if (nt == 5) return launch_sweep_fused_nt<T, true, 5>(L, uin, f, uout, rq, ry, smem, s);
    if (nt == 9) return launch_sweep_fused_nt<T, true, 9>(L, uin, f, uout, rq, ry, smem, s);
    return launch_sweep_fused_nt<T, true, 0>(L, uin, f, uout, rq, ry, smem, s);
  }
  if (nt == 5) return launch_sweep_fused_nt<T, false, 5>(L, uin, f, uout, rq, ry, smem, s);
  if (nt == 9) return launch_sweep_fused_nt<T, false, 9>(L, uin, f, uout, rq, ry, smem, s);
  return launch_sweep_fused_nt<T, false, 0>(L, uin, f, uout, rq, ry, smem, s);
}

template <typename T>
cudaError_t launch_jacobi(const LevelPair<T>& L, bool exact, const T* uin, const T* f, T* uout,
                          cudaStream_t s) {
  if (exact) k_jacobi<T, true><<<grid_of(L.h), dim3(kBX, kBY), 0, s>>>(L.d, uin, f, uout);
  else k_jacobi<T, false><<<grid_of(L.h), dim3(kBX, kBY), 0, s>>>(L.d, uin, f, uout);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_apply(const LevelPair<T>& L, bool exact, const T* u, T* out, cudaStream_t s) {
  if (exact) k_apply<T, true><<<grid_of(L.h), dim3(kBX, kBY), 0, s>>>(L.d, u, out);
  else k_apply<T, false><<<grid_of(L.h), dim3(kBX, kBY), 0, s>>>(L.d, u, out);
  return cudaGetLastError();
}

template <typename T, int NT>
cudaError_t launch_residual_nt(const LevelPair<T>& L, bool exact, const T* u, const T* f, T* d, cudaStream_t s) {
  dim3 g = grid_of(L.h);
  g.y = (L.h.rows + kBY * RowsPer<T>::value - 1) / (kBY * RowsPer<T>::value);
  const dim3 b(kBX, kBY);
  if (L.h.per) {
    if (exact) k_residual_nt<T, true, NT, true><<<g, b, 0, s>>>(L.d, u, f, d);
    else k_residual_nt<T, false, NT, true><<<g, b, 0, s>>>(L.d, u, f, d);
  } else {
    if (exact) k_residual_nt<T, true, NT, false><<<g, b, 0, s>>>(L.d, u, f, d);
    else k_residual_nt<T, false, NT, false><<<g, b, 0, s>>>(L.d, u, f, d);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_residual(const LevelPair<T>& L, bool exact, const T* u, const T* f, T* d,
                            cudaStream_t s) {
  const int ntf = fast_nt(L.h);
  if (ntf == 5) return launch_residual_nt<T, 5>(L, exact, u, f, d, s);
  if (ntf == 9) return launch_residual_nt<T, 9>(L, exact, u, f, d, s);
  dim3 g = grid_of(L.h);
  const int by = gen_block_rows(L.h, g.x);
  g.y = (L.h.rows + by - 1) / by;
  const bool deep = sizeof(T) == 4 && L.h.rows < kGenDeepRows;
  if (deep) {
    if (exact) k_residual_gen<T, true, true><<<g, dim3(kBX, by), 0, s>>>(L.d, u, f, d);
    else k_residual_gen<T, false, true><<<g, dim3(kBX, by), 0, s>>>(L.d, u, f, d);
  } else {
    if (exact) k_residual_gen<T, true, false><<<g, dim3(kBX, by), 0, s>>>(L.d, u, f, d);
    else k_residual_gen<T, false, false><<<g, dim3(kBX, by), 0, s>>>(L.d, u, f, d);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restrict(const LevelPair<T>& Lf, const LevelPair<T>& Lc, int transfer, bool exact,
                            const T* d, T* fc, cudaStream_t s, T* tc) {
  dim3 g = grid_of(Lc.h);
  const dim3 b(kBX, kBY);
  if (transfer != kStandardCubic && Lc.h.rows >= kTransferRowsMinLevelRows) {
    g.y = (Lc.h.rows + kBY * kTransferRows - 1) / (kBY * kTransferRows);
#define NSMG_RESTRICT(E, P) k_restrict<T, E, P, kTransferRows><<<g, b, 0, s>>>(Lf.d, Lc.d, transfer, d, fc, tc)
    if (Lf.h.per) {
      if (exact) NSMG_RESTRICT(true, true);
      else NSMG_RESTRICT(false, true);
    } else {
      if (exact) NSMG_RESTRICT(true, false);
      else NSMG_RESTRICT(false, false);
    }
#undef NSMG_RESTRICT
    return cudaGetLastError();
  }
  if (transfer == kStandardCubic) {
    if (Lf.h.per) {
      if (exact) k_restrict_cubic<T, true, true><<<g, b, 0, s>>>(Lf.d, Lc.d, d, fc, tc);
      else k_restrict_cubic<T, false, true><<<g, b, 0, s>>>(Lf.d, Lc.d, d, fc, tc);
    } else {
      if (exact) k_restrict_cubic<T, true, false><<<g, b, 0, s>>>(Lf.d, Lc.d, d, fc, tc);
      else k_restrict_cubic<T, false, false><<<g, b, 0, s>>>(Lf.d, Lc.d, d, fc, tc);
    }
  } else if (Lf.h.per) {
    if (exact) k_restrict<T, true, true, 1><<<g, b, 0, s>>>(Lf.d, Lc.d, transfer, d, fc, tc);
    else k_restrict<T, false, true, 1><<<g, b, 0, s>>>(Lf.d, Lc.d, transfer, d, fc, tc);
  } else {
    if (exact) k_restrict<T, true, false, 1><<<g, b, 0, s>>>(Lf.d, Lc.d, transfer, d, fc, tc);
    else k_restrict<T, false, false, 1><<<g, b, 0, s>>>(Lf.d, Lc.d, transfer, d, fc, tc);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong_add(const LevelPair<T>& Lf, const LevelPair<T>& Lc, int transfer,
                               bool exact, T* uf, const T* vc, cudaStream_t s, const T* uin) {
  const dim3 b(kBX, kBY);
  const T* ui = uin ? uin : uf;
  if (transfer != kStandardCubic && Lf.h.kind == kAxis && Lf.h.rows >= kTransferRowsMinLevelRows) {
    const dim3 g((Lf.h.n / 2 + 1 + kBX - 1) / kBX, (Lf.h.rows + kBY * kTransferRows - 1) / (kBY * kTransferRows));
#define NSMG_PROLONG(E, P) k_prolong_add<T, E, P, kTransferRows, true><<<g, b, 0, s>>>(Lf.d, Lc.d, transfer, ui, uf, vc)
    if (Lc.h.per) {
      if (exact) NSMG_PROLONG(true, true);
      else NSMG_PROLONG(false, true);
    } else {
      if (exact) NSMG_PROLONG(true, false);
      else NSMG_PROLONG(false, false);
    }
#undef NSMG_PROLONG
    return cudaGetLastError();
  }
  const dim3 g = grid_of(Lf.h);
  if (transfer == kStandardCubic) {
    if (Lc.h.per) {
      if (exact) k_prolong_cubic<T, true, true><<<g, b, 0, s>>>(Lf.d, Lc.d, ui, uf, vc);
      else k_prolong_cubic<T, false, true><<<g, b, 0, s>>>(Lf.d, Lc.d, ui, uf, vc);
    } else {
      if (exact) k_prolong_cubic<T, true, false><<<g, b, 0, s>>>(Lf.d, Lc.d, ui, uf, vc);
      else k_prolong_cubic<T, false, false><<<g, b, 0, s>>>(Lf.d, Lc.d, ui, uf, vc);
    }
  } else if (Lc.h.per) {
    if (exact) k_prolong_add<T, true, true, 1, false><<<g, b, 0, s>>>(Lf.d, Lc.d, transfer, ui, uf, vc);
    else k_prolong_add<T, false, true, 1, false><<<g, b, 0, s>>>(Lf.d, Lc.d, transfer, ui, uf, vc);
  } else {
    if (exact) k_prolong_add<T, true, false, 1, false><<<g, b, 0, s>>>(Lf.d, Lc.d, transfer, ui, uf, vc);
    else k_prolong_add<T, false, false, 1, false><<<g, b, 0, s>>>(Lf.d, Lc.d, transfer, ui, uf, vc);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarsest_dense(const DenseCoarse<T>& C, const LevelPair<T>& L, bool exact, const T* f, T* y, T* u,
                                  cudaStream_t s) {
  const int threads = std::min(1024, (C.m + 31) / 32 * 32);
  if (exact) k_coarsest_dense<T, true><<<1, threads, 0, s>>>(C, L.d, f, y, u);
  else k_coarsest_dense<T, false><<<1, threads, 0, s>>>(C, L.d, f, y, u);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarsest(int64_t idx, T a, int zero_mean, const T* f, T* u, cudaStream_t s) {
  k_coarsest<T><<<1, 32, 0, s>>>(idx, a, zero_mean, f, u);
  return cudaGetLastError();
}

// Blocks of a kernel resident on the whole GPU at once (256-thread blocks), looked up
// once per kernel.
template <auto KERNEL>
int resident_blocks() {
  static const int v = [] {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, KERNEL, kBX * kBY, 0) != cudaSuccess || nb < 1) {
      cudaGetLastError();
      nb = 1;
    }
    return nb * sm_count();
  }();
  return v;
}

// Partial sums a norm reduction of level L may need: at most kMaxPartials.
template <typename T>
int resnorm_blocks(const LevelPair<T>& L) {
  const dim3 g = norm_grid(L.h);
  return (int)(g.x * g.y);
}

template <typename T>
cudaError_t launch_resnorm(const LevelPair<T>& L, bool exact, const T* u, const T* f,
                           double* partial, double* out, cudaStream_t s) {
  const dim3 g = norm_grid(L.h);
  const int ty = (int)grid_of(L.h).y;
  if (exact) k_resnorm_partial<T, true><<<g, dim3(kBX, kBY), 0, s>>>(L.d, u, f, partial, ty);
  else k_resnorm_partial<T, false><<<g, dim3(kBX, kBY), 0, s>>>(L.d, u, f, partial, ty);
  k_sum_partials<<<1, dim3(kBX, kBY), 0, s>>>(partial, (int)(g.x * g.y), out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_first_half_zero(const LevelPair<T>& L, const T* f, T* t, int red, cudaStream_t s) {
  k_first_half_zero<T><<<grid_of(L.h), dim3(kBX, kBY), 0, s>>>(L.d, f, t, red);
  return cudaGetLastError();
}

template <typename T, bool EXACT, int NT>
cudaError_t launch_resnorm_red_as(const LevelPair<T>& L, const T* u, const T* f, T* uout, int red, double* partial,
                                  double* out, cudaStream_t s) {
  const dim3 t = grid_of(L.h);
  const int tiles = (int)(t.x * t.y);
  const int blocks = std::min({tiles, kMaxPartials, resident_blocks<k_resnorm_red<T, EXACT, NT>>()});
  k_resnorm_red<T, EXACT, NT><<<blocks, dim3(kBX, kBY), 0, s>>>(L.d, u, f, uout, red, partial, (int)t.x, tiles);
  k_sum_partials<<<1, dim3(kBX, kBY), 0, s>>>(partial, blocks, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_resnorm_red(const LevelPair<T>& L, bool exact, const T* u, const T* f, T* uout, int red,
                               double* partial, double* out, cudaStream_t s) {
  const int nt = L.h.kind == kAxis ? fast_nt(L.h) : 0;
  if (nt == 9)
    return exact ? launch_resnorm_red_as<T, true, 9>(L, u, f, uout, red, partial, out, s)
                 : launch_resnorm_red_as<T, false, 9>(L, u, f, uout, red, partial, out, s);
  if (nt == 5)
    return exact ? launch_resnorm_red_as<T, true, 5>(L, u, f, uout, red, partial, out, s)
                 : launch_resnorm_red_as<T, false, 5>(L, u, f, uout, red, partial, out, s);
  return exact ? launch_resnorm_red_as<T, true, 0>(L, u, f, uout, red, partial, out, s)
               : launch_resnorm_red_as<T, false, 0>(L, u, f, uout, red, partial, out, s);
}

template <typename T>
cudaError_t launch_sumsq(const LevelPair<T>& L, const T* f, double* partial, double* out,
                         cudaStream_t s) {
  const dim3 g = norm_grid(L.h);
  k_sumsq_partial<T><<<g, dim3(kBX, kBY), 0, s>>>(L.d, f, partial, (int)grid_of(L.h).y);
  k_sum_partials<<<1, dim3(kBX, kBY), 0, s>>>(partial, (int)(g.x * g.y), out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_copy_boundary(const LevelPair<T>& L, const T* src, T* dst, cudaStream_t s) {
  const int n = L.h.n;
  k_copy_boundary<T><<<(n + 1 + 255) / 256, 256, 0, s>>>(n, L.h.pitch, src, dst);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_zero_boundary(const LevelPair<T>& L, T* u, cudaStream_t s) {
  const int n = L.h.n;
  k_zero_boundary<T><<<(n + 1 + 255) / 256, 256, 0, s>>>(n, L.h.pitch, u);
  return cudaGetLastError();
}

template <bool EXACT, int NT>
cudaError_t launch_ir_residual_as(const LevelPair<double>& L, const double* u, const double* f,
                                  const LevelPair<float>& L32, float* r32, double scale, double* partial, double* out,
                                  cudaStream_t s, int bf16, float* t32) {
  const dim3 t = grid_of(L.h);
  const int tiles = (int)(t.x * t.y);
  const int blocks = std::min({tiles, kMaxPartials, resident_blocks<k_ir_residual<EXACT, NT>>()});
  k_ir_residual<EXACT, NT><<<blocks, dim3(kBX, kBY), 0, s>>>(L.d, u, f, r32, scale, partial, (int)t.x, tiles, bf16,
                                                             L32.d, t32);
  k_sum_partials<<<1, dim3(kBX, kBY), 0, s>>>(partial, blocks, out);
  return cudaGetLastError();
}

cudaError_t launch_ir_residual(const LevelPair<double>& L, bool exact, const double* u, const double* f,
                               const LevelPair<float>& L32, float* r32, double scale, double* partial,
                               double* out, cudaStream_t s, int bf16, float* t32) {
  const int ntf = fast_nt(L.h);
  if (ntf == 9)
    return exact ? launch_ir_residual_as<true, 9>(L, u, f, L32, r32, scale, partial, out, s, bf16, t32)
                 : launch_ir_residual_as<false, 9>(L, u, f, L32, r32, scale, partial, out, s, bf16, t32);
  if (ntf == 5)
    return exact ? launch_ir_residual_as<true, 5>(L, u, f, L32, r32, scale, partial, out, s, bf16, t32)
                 : launch_ir_residual_as<false, 5>(L, u, f, L32, r32, scale, partial, out, s, bf16, t32);
  return exact ? launch_ir_residual_as<true, 0>(L, u, f, L32, r32, scale, partial, out, s, bf16, t32)
               : launch_ir_residual_as<false, 0>(L, u, f, L32, r32, scale, partial, out, s, bf16, t32);
}

cudaError_t launch_ir_update(const LevelPair<double>& L, const LevelPair<float>& L32, double* u, const float* e,
                             double inv_scale, cudaStream_t s) {
  dim3 g = grid_of(L.h);
  g.y = (L.h.rows + kBY * kTransferRows - 1) / (kBY * kTransferRows);
  k_ir_update<<<g, dim3(kBX, kBY), 0, s>>>(L.d, L32.h.pitch, u, e, inv_scale);
  return cudaGetLastError();
}

template <typename T, bool EXACT>
cudaError_t launch_tail_impl(int ctas, const TailDesc<T>* desc, const int4* prog, int nops, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(kTailThreads);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = ctas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_tail<T, EXACT>, desc, prog, nops);
}

// Largest cluster the device can co-schedule for the tail kernel: 16 CTAs
// (non-portable size) when available, else 8, else 1.
template <typename T, bool EXACT>
int tail_ctas_impl() {
  cudaFuncSetAttribute(k_tail<T, EXACT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  for (int c : {16, 8, 4, 2}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c);
    cfg.blockDim = dim3(kTailThreads);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, k_tail<T, EXACT>, &cfg) == cudaSuccess && clusters > 0) return c;
    cudaGetLastError();
  }
  return 1;
}

template <typename T>
int tail_ctas(bool exact) {
  return exact ? tail_ctas_impl<T, true>() : tail_ctas_impl<T, false>();
}

template <typename T>
cudaError_t launch_tail(int ctas, const TailDesc<T>* desc, const int4* prog, int nops, bool exact, cudaStream_t s) {
  return exact ? launch_tail_impl<T, true>(ctas, desc, prog, nops, s)
               : launch_tail_impl<T, false>(ctas, desc, prog, nops, s);
}

template <typename T>
cudaError_t launch_batch_step(int op, const BatchLevel<T>* entries, const int* prefix, int ne, int total_tiles,
                              int rpt, const int* active, bool exact, cudaStream_t s) {
  if (ne <= 0) return cudaSuccess;
  if (op == kBCoarsest) {
    k_batch_coarsest<T><<<(ne + 127) / 128, 128, 0, s>>>(entries, ne, active);
    return cudaGetLastError();
  }
  if (op == kBCoarsestDense) {
    if (exact) k_batch_coarsest_dense<T, true><<<ne, 256, 0, s>>>(entries, active);
    else k_batch_coarsest_dense<T, false><<<ne, 256, 0, s>>>(entries, active);
    return cudaGetLastError();
  }
  if (total_tiles <= 0) return cudaSuccess;
  const dim3 blk(kBX, kBY);
#define NSMG_BSTEP(R)                                                                                   \
  if (rpt == R) {                                                                                       \
    if (exact) k_batch_step<T, true, R><<<total_tiles, blk, 0, s>>>(op, entries, prefix, ne, active);  \
    else k_batch_step<T, false, R><<<total_tiles, blk, 0, s>>>(op, entries, prefix, ne, active);       \
    return cudaGetLastError();                                                                          \
  }
  NSMG_BSTEP(1)
  NSMG_BSTEP(2)
  NSMG_BSTEP(4)
#undef NSMG_BSTEP
  return cudaErrorInvalidValue;
}

cudaError_t launch_batch_norms(int mode, const BatchLevel<double>* entries, const int* prefix, int ne,
                               int total_tiles, const int* active, const double* scale, bool exact,
                               double* partial, double* norm2, cudaStream_t s) {
  if (ne <= 0 || total_tiles <= 0) return cudaSuccess;
  if (exact) k_batch_norm_partial<true><<<total_tiles, dim3(kBX, kBY), 0, s>>>(mode, entries, prefix, ne, active, scale, partial);
  else k_batch_norm_partial<false><<<total_tiles, dim3(kBX, kBY), 0, s>>>(mode, entries, prefix, ne, active, scale, partial);
  k_batch_norm_sum<<<ne, dim3(kBX, kBY), 0, s>>>(entries, prefix, active, partial, norm2);
  return cudaGetLastError();
}

cudaError_t launch_batch_ir_update(const BatchLevel<double>* entries, const int* prefix, int ne, int total_tiles,
                                   const int* active, const double* scale, cudaStream_t s) {
  if (ne <= 0 || total_tiles <= 0) return cudaSuccess;
  k_batch_ir_update<<<total_tiles, dim3(kBX, kBY), 0, s>>>(entries, prefix, ne, active, scale);
  return cudaGetLastError();
}

template <typename T>
size_t tail_smem_bytes(int sm_elems, int nst) {
  return TailStencil::base<T>(sm_elems) + (size_t)nst * kMaxTerms * (sizeof(T) + 2 * sizeof(int));
}

template <typename T>
cudaError_t launch_tail_smem(const TailDesc<T>* desc, int sm_elems, int nst, const int4* prog, int nops, bool exact,
                             cudaStream_t s) {
  const size_t bytes = tail_smem_bytes<T>(sm_elems, nst);
  if (bytes > kTailSmemMaxBytes) return cudaErrorInvalidValue;
  const void* fn = exact ? (const void*)k_tail_smem<T, true> : (const void*)k_tail_smem<T, false>;
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (exact) k_tail_smem<T, true><<<1, kTailThreads, bytes, s>>>(desc, prog, nops);
  else k_tail_smem<T, false><<<1, kTailThreads, bytes, s>>>(desc, prog, nops);
  return cudaGetLastError();
}

#define NSMG_INSTANTIATE(T)                                                                           \
  template cudaError_t launch_half_sweep<T>(const LevelPair<T>&, bool, const T*, const T*, T*, int,   \
                                            cudaStream_t);                                            \
  template cudaError_t launch_jacobi<T>(const LevelPair<T>&, bool, const T*, const T*, T*,            \
                                        cudaStream_t);                                                \
  template cudaError_t launch_apply<T>(const LevelPair<T>&, bool, const T*, T*, cudaStream_t);        \
  template cudaError_t launch_residual<T>(const LevelPair<T>&, bool, const T*, const T*, T*,          \
                                          cudaStream_t);                                              \
  template cudaError_t launch_restrict<T>(const LevelPair<T>&, const LevelPair<T>&, int, bool,        \
                                          const T*, T*, cudaStream_t, T*);                            \
  template cudaError_t launch_prolong_add<T>(const LevelPair<T>&, const LevelPair<T>&, int, bool, T*, \
                                             const T*, cudaStream_t, const T*);                       \
  template cudaError_t launch_sweep_fused<T>(const LevelPair<T>&, bool, const T*, const T*, T*, cudaStream_t); \
  template cudaError_t launch_coarsest<T>(int64_t, T, int, const T*, T*, cudaStream_t);                    \
  template cudaError_t launch_coarsest_dense<T>(const DenseCoarse<T>&, const LevelPair<T>&, bool, const T*, T*, T*, \
                                                cudaStream_t);                                                     \
  template int resnorm_blocks<T>(const LevelPair<T>&);                                                \
  template cudaError_t launch_resnorm<T>(const LevelPair<T>&, bool, const T*, const T*, double*,     \
                                         double*, cudaStream_t);                                      \
  template cudaError_t launch_first_half_zero<T>(const LevelPair<T>&, const T*, T*, int, cudaStream_t); \
  template cudaError_t launch_resnorm_red<T>(const LevelPair<T>&, bool, const T*, const T*, T*, int,  \
                                             double*, double*, cudaStream_t);                         \
  template cudaError_t launch_sumsq<T>(const LevelPair<T>&, const T*, double*, double*, cudaStream_t); \
  template cudaError_t launch_zero_boundary<T>(const LevelPair<T>&, T*, cudaStream_t);                \
  template cudaError_t launch_copy_boundary<T>(const LevelPair<T>&, const T*, T*, cudaStream_t);      \
  template cudaError_t launch_batch_step<T>(int, const BatchLevel<T>*, const int*, int, int, int, const int*, bool, \
                                            cudaStream_t);                                             \
  template int tail_ctas<T>(bool);                                                                    \
  template cudaError_t launch_tail_smem<T>(const TailDesc<T>*, int, int, const int4*, int, bool, cudaStream_t); \
  template size_t tail_smem_bytes<T>(int, int);                                                       \
  template cudaError_t launch_tail<T>(int, const TailDesc<T>*, const int4*, int, bool, cudaStream_t);

NSMG_INSTANTIATE(double)
NSMG_INSTANTIATE(float)

}  // namespace nsmg

// ---------------------------------------------------------------------------
// Relative residual of the finest level without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// residual norm: real-time loops that must not hit the implicit device
// synchronisation of cudaMalloc / cudaFree, or hosts that hand the library a fixed
// memory budget (or an arena they manage) and forbid allocation after set-up. For
// them the partial sums
// of the reduction live in a file-scope device array instead of in memory obtained
// from the allocator: every GPU that loads this library holds
// kStaticNormPartials x 2 doubles (32 KB) until the process exits.
#include <mutex>

#include "../../include/nsmg.h"

namespace nsmg {

// Finest-level FP64 description of a handle and its evaluation order (hierarchy.cu).
const LevelPair<double>* finest_level_fp64(const mg_handle* h, bool* exact);

namespace {

constexpr int kStaticNormPartials = 2048;  // blocks per reduction (sum of squares of d and of f)
static __device__ __align__(256) double g_static_norm_scratch[2 * kStaticNormPartials];

// Block-wide sums of two doubles (blockDim = 256).
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double pa[32], pb[32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  if (lane == 0) {
    pa[warp] = a;
    pb[warp] = b;
  }
  __syncthreads();
  const int nw = (blockDim.x * blockDim.y) >> 5;
  a = tid < nw ? pa[tid] : 0.0;
  b = tid < nw ? pb[tid] : 0.0;
  if (warp == 0)
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
}

// Block (bx, by) reduces the 32 x 8 tiles (bx, by), (bx, by + gridDim.y), ... into
// scratch[b] (sum of d^2) and scratch[kStaticNormPartials + b] (sum of f^2).
template <bool EXACT>
__global__ void k_resnorm_static(const LevelDev<double>* __restrict__ Lp, const double* __restrict__ u,
                                 const double* __restrict__ f, double* __restrict__ scratch, int tiles_y) {
  const LevelDev<double>& L = *Lp;
  double sd = 0.0, sf = 0.0;
  const int q = blockIdx.x * kBX + threadIdx.x;
  for (int ty = blockIdx.y; ty < tiles_y; ty += gridDim.y) {
    const int j = ty * kBY + threadIdx.y;
    if (j >= L.rows || q >= L.cols) continue;
    const int i = L.kind == kRot ? 2 * q + (j & 1) : q;
    if (!interior(L, i, j)) continue;
    const int64_t at = sidx(L, i, j);
    const double d = Arith<double>::sub(f[at], apply_at<double, EXACT>(L, u, i, j, at, nullptr));
    sd += d * d;
    sf += f[at] * f[at];
  }
  block_sum2(sd, sf);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    const int b = blockIdx.y * gridDim.x + blockIdx.x;
    scratch[b] = sd;
    scratch[kStaticNormPartials + b] = sf;
  }
}

// One block: add the `count` partials of each sum in a fixed order; write
// sqrt(sum d^2) / sqrt(sum f^2) to *out.
__global__ void k_static_norm_finish(const double* __restrict__ scratch, int count, double* __restrict__ out) {
  double a = 0.0, b = 0.0;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  for (int k = tid; k < count; k += blockDim.x * blockDim.y) {
    a += scratch[k];
    b += scratch[kStaticNormPartials + k];
  }
  block_sum2(a, b);
  if (tid == 0) *out = sqrt(a) / sqrt(b);
}

// Device address of g_static_norm_scratch on each device, looked up once per device
// with that device current. The name is only a host-side stand-in for the array.
std::mutex g_static_norm_mu;
double* g_static_norm_ptr[64] = {};

cudaError_t static_norm_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_static_norm_mu);
  if (!g_static_norm_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_norm_scratch);
    if (e != cudaSuccess) return e;
    g_static_norm_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_static_norm_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace nsmg

extern "C" mg_status mg_rel_residual_static(mg_handle* h, const double* u, const double* f, double* rel_res_dev,
                                            void* stream) {
  using namespace nsmg;
  bool exact = true;
  const LevelPair<double>* L = finest_level_fp64(h, &exact);
  if (!L || !u || !f || !rel_res_dev) return MG_ERR_INVALID;
  const int tiles_x = (L->h.cols + kBX - 1) / kBX;
  const int tiles_y = (L->h.rows + kBY - 1) / kBY;
  if (tiles_x > kStaticNormPartials) return MG_ERR_UNSUPPORTED;  // grid wider than the scratch array
  const int gy = std::max(1, std::min(tiles_y, kStaticNormPartials / tiles_x));
  double* scratch = nullptr;
  if (static_norm_scratch(&scratch) != cudaSuccess) return MG_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const dim3 grid(tiles_x, gy);
  if (exact) k_resnorm_static<true><<<grid, dim3(kBX, kBY), 0, s>>>(L->d, u, f, scratch, tiles_y);
  else k_resnorm_static<false><<<grid, dim3(kBX, kBY), 0, s>>>(L->d, u, f, scratch, tiles_y);
  k_static_norm_finish<<<1, dim3(kBX, kBY), 0, s>>>(scratch, tiles_x * gy, rel_res_dev);
  return cudaGetLastError() == cudaSuccess ? MG_OK : MG_ERR_CUDA;
}
