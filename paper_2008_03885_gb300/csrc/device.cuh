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

// One class term by a single 16-byte load.
template <typename T>
__device__ __forceinline__ ClassTerm<T> load_term(const ClassTerm<T>* p) {
  const int4 w = __ldg(reinterpret_cast<const int4*>(p));
  ClassTerm<T> t;
  if (sizeof(T) == 8) {
    t.c = (T)__hiloint2double(w.y, w.x);
    t.dx = w.z;
    t.dy = w.w;
  } else {
    t.c = (T)__int_as_float(w.x);
    t.dx = w.y;
    t.dy = w.z;
  }
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
  T s;
  if (fast_node(L, i, j)) {
    const int32_t* dl = L.delta[L.kind == kRot ? (i & 1) : 0];
    s = Arith<T>::mul(L.c[0], u[at + dl[0]]);
#pragma unroll CU
    for (int k = 1; k < L.nt; ++k) s = madd<T, EXACT>(s, L.c[k], u[at + dl[k]]);
    if (wd) *wd = L.wd;
  } else {
    const int cl = class_of(L, i, j);
    const int2 e = L.cls[cl];
    const ClassTerm<T>* tt = L.terms + e.x;
    s = T(0);
#pragma unroll CU
    for (int k = 0; k < e.y; ++k) {
      const ClassTerm<T> t = load_term(tt + k);
      const T x = u[sidx(L, i + t.dx, j + t.dy)];
      s = k == 0 ? Arith<T>::mul(t.c, x) : madd<T, EXACT>(s, t.c, x);
    }
    if (wd) *wd = L.cls_wd[cl];
  }
  return s;
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

template <typename T, bool EXACT, int NT>
__device__ __forceinline__ T apply_fast(const T (&c)[NT], const int (&dl)[NT], const T* __restrict__ u,
                                        int64_t at) {
  T s = Arith<T>::mul(c[0], u[at + dl[0]]);
#pragma unroll
  for (int k = 1; k < NT; ++k) s = madd<T, EXACT>(s, c[k], u[at + dl[k]]);
  return s;
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
