// Device helpers shared by the kernel translation units: rounding-mode arithmetic,
// level geometry (storage index, colour, boundary class, fast-node test) and the
// stencil sums in the fixed evaluation order (see kernels.cu).
#pragma once

#include <cuda_bf16.h>

#include "levels.h"

namespace nsmg {
namespace {


constexpr int kBX = 32, kBY = 8;

// Minimum resident 256-thread blocks per SM requested from the compiler: FP32 stencil
// kernels are memory-latency bound and gain from full occupancy (8 blocks: 32
// registers); FP64 kernels are bound by the FP64 pipe and keep their registers.
template <typename T>
struct MinBlocks {
  static constexpr int value = sizeof(T) == 4 ? 8 : 4;
};

template <typename T>
struct Arith;
template <>
struct Arith<double> {
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }
  static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
};
template <>
struct Arith<float> {
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float fma(float a, float b, float c) { return fmaf(a, b, c); }
  static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
};

// One class term by a single 16-byte load; `start` is set on the first term of a group
// of equal coefficients (the flag travels in dx, see kTermStart).
template <typename T>
struct Term {
  T c;
  int dx, dy;
  bool start;
};
template <typename T>
__device__ __forceinline__ Term<T> load_term(const ClassTerm<T>* p) {
  const int4 w = __ldg(reinterpret_cast<const int4*>(p));
  Term<T> t;
  int dx;
  if (sizeof(T) == 8) {
    t.c = (T)__hiloint2double(w.y, w.x);
    dx = w.z;
    t.dy = w.w;
  } else {
    t.c = (T)__int_as_float(w.x);
    dx = w.y;
    t.dy = w.z;
  }
  t.start = dx >= (kTermStart >> 1);
  t.dx = t.start ? dx - kTermStart : dx;
  return t;
}

// Hint: bring the line holding *p into L2, so that the loads issued later wait on L2
// rather than DRAM (more bytes in flight than the registers of a thread allow).
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// s + c * x in the chosen rounding mode.
// Value as stored on a level: FP32 levels of the bfloat16 storage trial round it.
template <typename T>
__device__ __forceinline__ T rnd(const LevelDev<T>& L, T v) {
  return v;
}
template <>
__device__ __forceinline__ float rnd<float>(const LevelDev<float>& L, float v) {
  return L.bf16 ? __bfloat162float(__float2bfloat16_rn(v)) : v;
}

template <typename T, bool EXACT>
__device__ __forceinline__ T madd(T s, T c, T x) {
  return EXACT ? Arith<T>::add(s, Arith<T>::mul(c, x)) : Arith<T>::fma(c, x, s);
}

// One operator row in the evaluation order: terms arrive in evaluation order (groups of
// equal coefficient, see LevelDev::c), `start` on the first term of each group.
// EXACT: sum_g c_g * (x_g1 + x_g2 + ...), the group sums and the outer sum left to right,
// every operation rounded separately. Otherwise one fused multiply-add per term, from
// the first product.
template <typename T, bool EXACT>
struct RowSum {
  T s = T(0);   // sum of the closed groups (EXACT) or running sum
  T g = T(0);   // open group's sum of values
  T cg = T(0);  // open group's coefficient
  bool any = false, open = false;
  __device__ __forceinline__ void add(T c, T x, bool start) {
    if (EXACT) {
      if (start) {
        close();
        g = x;
        cg = c;
        open = true;
      } else {
        g = Arith<T>::add(g, x);
      }
    } else {
      s = any ? Arith<T>::fma(c, x, s) : Arith<T>::mul(c, x);
      any = true;
    }
  }
  __device__ __forceinline__ void close() {
    if (EXACT && open) {
      const T p = Arith<T>::mul(cg, g);
      s = any ? Arith<T>::add(s, p) : p;
      any = true;
      open = false;
    }
  }
  __device__ __forceinline__ T value() {
    close();
    return s;
  }
};

__device__ __forceinline__ bool gbit(const uint32_t* m, int k) { return (m[k >> 5] >> (k & 31)) & 1u; }

template <typename T>
__device__ __forceinline__ int64_t sidx(const LevelDev<T>& L, int i, int j) {
  return (int64_t)j * L.pitch + (L.kind == kRot ? (i >> 1) : i);
}

// Lattice coordinates of the thread's storage element; false if outside storage.
template <typename T>
__device__ __forceinline__ bool thread_node(const LevelDev<T>& L, int& i, int& j) {
  const int q = blockIdx.x * kBX + threadIdx.x;
  j = blockIdx.y * blockDim.y + threadIdx.y;
  if (j >= L.rows || q >= L.cols) return false;
  i = L.kind == kRot ? 2 * q + (j & 1) : q;
  return true;
}

template <typename T>
__device__ __forceinline__ bool interior(const LevelDev<T>& L, int i, int j) {
  return i >= L.lo && i < L.n && j >= L.lo && j < L.n;
}

template <typename T>
__device__ __forceinline__ bool is_red(const LevelDev<T>& L, int i, int j) {
  return L.kind == kRot ? (i & 1) : ((i + j) & 1);
}

// Class index of a node that is not a fast node.
template <typename T>
__device__ __forceinline__ int class_of(const LevelDev<T>& L, int i, int j) {
  if (L.small) return j * L.clsw + i;
  const int e = L.n - L.per;  // last lattice index a fast stencil may reach
  const int cx = i < L.rx ? i : (i > e - L.rx ? 2 * L.rx - (e - i) : L.rx);
  const int cy = j < L.ry ? j : (j > e - L.ry ? 2 * L.ry - (e - j) : L.ry);
  return cy * L.clsw + cx;
}

template <typename T>
__device__ __forceinline__ bool fast_node(const LevelDev<T>& L, int i, int j) {
  return i >= L.rx && i <= L.fxe && j >= L.ry && j <= L.fye;
}

// omega / a_pp of node (i, j).
template <typename T>
__device__ __forceinline__ T node_wd(const LevelDev<T>& L, int i, int j) {
  return fast_node(L, i, j) ? L.wd : L.cls_wd[class_of(L, i, j)];
}

// First half-sweep value from u = 0 (see k_first_half_zero): 0 + f omega / a_pp.
template <typename T>
__device__ __forceinline__ T relax_from_zero(T f, T wd) {
  return Arith<T>::add(T(0), Arith<T>::mul(f, wd));
}

// (L u)(i, j) and the node's omega / a_pp.
// CU: unroll factor of the boundary-class term loop (its loads then run ahead of the
// ordered sum); 1 in the register-tight NT kernels.
template <typename T, bool EXACT, int CU = 4>
__device__ __forceinline__ T apply_at(const LevelDev<T>& L, const T* __restrict__ u, int i, int j,
                                      int64_t at, T* wd) {
  RowSum<T, EXACT> acc;
  if (fast_node(L, i, j)) {
    const int32_t* dl = L.delta[L.kind == kRot ? (i & 1) : 0];
#pragma unroll CU
    for (int k = 0; k < L.nt; ++k) acc.add(L.c[k], u[at + dl[k]], gbit(L.gmask, k));
    if (wd) *wd = L.wd;
  } else {
    const int cl = class_of(L, i, j);
    const int2 e = L.cls[cl];
    const ClassTerm<T>* tt = L.terms + e.x;
#pragma unroll CU
    for (int k = 0; k < e.y; ++k) {
      const Term<T> t = load_term(tt + k);
      acc.add(t.c, u[sidx(L, i + t.dx, j + t.dy)], t.start);
    }
    if (wd) *wd = L.cls_wd[cl];
  }
  return acc.value();
}

// New value of node (i, j) after one relaxation: u + (f - L u) * omega / a_pp.
template <typename T, bool EXACT, int CU = 4>
__device__ __forceinline__ T relax_value(const LevelDev<T>& L, const T* __restrict__ uin,
                                         const T* __restrict__ f, int i, int j, int64_t at) {
  T wd;
  const T s = apply_at<T, EXACT, CU>(L, uin, i, j, at, &wd);
  const T r = Arith<T>::sub(f[at], s);
  return EXACT ? Arith<T>::add(uin[at], Arith<T>::mul(r, wd)) : Arith<T>::fma(r, wd, uin[at]);
}

// ---- specialised fast path: NT-point stencils with coefficients in registers and
// kRows rows per thread (same arithmetic as apply_at / relax_value) --------------
// Rows per thread of the 5/9-point kernels (2 and 4 measured equal for FP32 on GB300).
template <typename T>
struct RowsPer {
  static constexpr int value = 4;
};

// The NT-term fast stencils come in fixed group shapes (checked on the host, see
// fast_groups_ok): 5 terms = four equal neighbours, then the centre; 9 terms = two
// groups of four, then the centre (fourth-order cross, first Galerkin stencils).
__host__ __device__ constexpr uint32_t fast_gmask(int nt) { return nt == 9 ? 0x111u : nt == 5 ? 0x11u : 0u; }

template <typename T, bool EXACT, int NT>
__device__ __forceinline__ T apply_fast(const T (&c)[NT], const int (&dl)[NT], const T* __restrict__ u,
                                        int64_t at) {
  if constexpr (EXACT && (NT == 5 || NT == 9)) {
    T g0 = u[at + dl[0]];
#pragma unroll
    for (int k = 1; k < 4; ++k) g0 = Arith<T>::add(g0, u[at + dl[k]]);
    T s = Arith<T>::mul(c[0], g0);
    if (NT == 9) {
      T g1 = u[at + dl[4]];
#pragma unroll
      for (int k = 5; k < 8; ++k) g1 = Arith<T>::add(g1, u[at + dl[k]]);
      s = Arith<T>::add(s, Arith<T>::mul(c[4], g1));
    }
    return Arith<T>::add(s, Arith<T>::mul(c[NT - 1], u[at + dl[NT - 1]]));
  } else {
    // (fused multiply-adds; the EXACT form of other term counts is never instantiated for
    // use: the launchers take the NT kernels only for 5 and 9 terms)
    T s = Arith<T>::mul(c[0], u[at + dl[0]]);
#pragma unroll
    for (int k = 1; k < NT; ++k) s = Arith<T>::fma(c[k], u[at + dl[k]], s);
    return s;
  }
}

template <typename T, bool EXACT, int NT>
__device__ __forceinline__ T relax_fast(const T (&c)[NT], const int (&dl)[NT], T wd, const T* __restrict__ uin,
                                        const T* __restrict__ f, int64_t at) {
  const T r = Arith<T>::sub(f[at], apply_fast<T, EXACT, NT>(c, dl, uin, at));
  return EXACT ? Arith<T>::add(uin[at], Arith<T>::mul(r, wd)) : Arith<T>::fma(r, wd, uin[at]);
}

// fast_node with the boundary kind fixed at compile time (the NT kernels run at the
// register limit; constant bounds keep the Dirichlet instantiation free of spills).
template <bool PER, typename T>
__device__ __forceinline__ bool fast_node_c(const LevelDev<T>& L, int i, int j) {
  const int e = L.n - (PER ? 1 : 0);
  return i >= L.rx && i <= e - L.rx && j >= L.ry && j <= e - L.ry;
}

}  // namespace
}  // namespace nsmg
