// Multigrid kernels for sm_103a: stencil application with boundary classes,
// red-black and Jacobi relaxation, residual, restriction, interpolation with
// correction, coarsest solve, and a deterministic residual-norm reduction.
//
// Evaluation order (EXACT = true): each sum starts from its first product and
// adds the following products in the order of the term list (sorted by (dy, dx)),
// every product and sum rounded separately (__dmul_rn / __dadd_rn keep nvcc from
// contracting them into FMAs). EXACT = false lets products fuse into FMAs.
#include <algorithm>
#include <cstdio>

#include "kernels.h"

namespace nsmg {
namespace {

constexpr int kBX = 32, kBY = 8;

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

// s + c * x in the chosen rounding mode.
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
  j = blockIdx.y * kBY + threadIdx.y;
  if (j >= L.rows || q >= L.cols) return false;
  i = L.kind == kRot ? 2 * q + (j & 1) : q;
  return true;
}

template <typename T>
__device__ __forceinline__ bool interior(const LevelDev<T>& L, int i, int j) {
  return i > 0 && i < L.n && j > 0 && j < L.n;
}

template <typename T>
__device__ __forceinline__ bool is_red(const LevelDev<T>& L, int i, int j) {
  return L.kind == kRot ? (i & 1) : ((i + j) & 1);
}

// Class index of a node that is not a fast node.
template <typename T>
__device__ __forceinline__ int class_of(const LevelDev<T>& L, int i, int j) {
  if (L.small) return j * L.clsw + i;
  const int cx = i < L.rx ? i : (i > L.n - L.rx ? 2 * L.rx - (L.n - i) : L.rx);
  const int cy = j < L.ry ? j : (j > L.n - L.ry ? 2 * L.ry - (L.n - j) : L.ry);
  return cy * L.clsw + cx;
}

template <typename T>
__device__ __forceinline__ bool fast_node(const LevelDev<T>& L, int i, int j) {
  return i >= L.rx && i <= L.n - L.rx && j >= L.ry && j <= L.n - L.ry;
}

// (L u)(i, j) and the node's omega / a_pp.
template <typename T, bool EXACT>
__device__ __forceinline__ T apply_at(const LevelDev<T>& L, const T* __restrict__ u, int i, int j,
                                      int64_t at, T* wd) {
  T s;
  if (fast_node(L, i, j)) {
    const int32_t* dl = L.delta[L.kind == kRot ? (i & 1) : 0];
    s = Arith<T>::mul(L.c[0], u[at + dl[0]]);
    for (int k = 1; k < L.nt; ++k) s = madd<T, EXACT>(s, L.c[k], u[at + dl[k]]);
    if (wd) *wd = L.wd;
  } else {
    const int cl = class_of(L, i, j);
    const int2 e = L.cls[cl];
    s = T(0);
    for (int k = 0; k < e.y; ++k) {
      const int t = e.x + k;
      const T x = u[sidx(L, i + L.tdx[t], j + L.tdy[t])];
      s = k == 0 ? Arith<T>::mul(L.tc[t], x) : madd<T, EXACT>(s, L.tc[t], x);
    }
    if (wd) *wd = L.cls_wd[cl];
  }
  return s;
}

template <typename T, bool EXACT>
__global__ void k_half_sweep(const LevelDev<T>* __restrict__ Lp, const T* __restrict__ uin,
                             const T* __restrict__ f, T* __restrict__ uout, int red) {
  const LevelDev<T>& L = *Lp;
  int i, j;
  if (!thread_node(L, i, j) || !interior(L, i, j)) return;
  const int64_t at = sidx(L, i, j);
  if (is_red(L, i, j) != red) {
    uout[at] = uin[at];
    return;
  }
  T wd;
  const T s = apply_at<T, EXACT>(L, uin, i, j, at, &wd);
  const T r = Arith<T>::sub(f[at], s);
  uout[at] = EXACT ? Arith<T>::add(uin[at], Arith<T>::mul(r, wd)) : Arith<T>::fma(r, wd, uin[at]);
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
  uout[at] = EXACT ? Arith<T>::add(uin[at], Arith<T>::mul(r, wd)) : Arith<T>::fma(r, wd, uin[at]);
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

template <typename T, bool EXACT>
__global__ void k_residual(const LevelDev<T>* __restrict__ Lp, const T* __restrict__ u,
                           const T* __restrict__ f, T* __restrict__ d) {
  const LevelDev<T>& L = *Lp;
  int i, j;
  if (!thread_node(L, i, j) || !interior(L, i, j)) return;
  const int64_t at = sidx(L, i, j);
  d[at] = Arith<T>::sub(f[at], apply_at<T, EXACT>(L, u, i, j, at, nullptr));
}

// Restriction terms (dx, dy) in fine-lattice units, sorted by (dy, dx), with weights.
struct RTerm {
  int dx, dy;
  double w;
};
__constant__ RTerm c_rterms_rb_axis[5] = {{0, -1, 0.125}, {-1, 0, 0.125}, {0, 0, 0.5}, {1, 0, 0.125}, {0, 1, 0.125}};
__constant__ RTerm c_rterms_rb_rot[5] = {{-1, -1, 0.125}, {1, -1, 0.125}, {0, 0, 0.5}, {-1, 1, 0.125}, {1, 1, 0.125}};
__constant__ RTerm c_rterms_std[9] = {{-1, -1, 0.0625}, {0, -1, 0.125}, {1, -1, 0.0625},
                                      {-1, 0, 0.125},   {0, 0, 0.25},   {1, 0, 0.125},
                                      {-1, 1, 0.0625},  {0, 1, 0.125},  {1, 1, 0.0625}};

template <typename T, bool EXACT>
__global__ void k_restrict(const LevelDev<T>* __restrict__ Lfp, const LevelDev<T>* __restrict__ Lcp,
                           int transfer, const T* __restrict__ d, T* __restrict__ fc) {
  const LevelDev<T>& Lf = *Lfp;
  const LevelDev<T>& Lc = *Lcp;
  int i, j;
  if (!thread_node(Lc, i, j) || !interior(Lc, i, j)) return;
  // fine-lattice position of the coarse node
  const int fi = transfer == kRbAxisToRot ? i : 2 * i;
  const int fj = transfer == kRbAxisToRot ? j : 2 * j;
  const RTerm* rt = transfer == kRbAxisToRot ? c_rterms_rb_axis
                    : transfer == kRbRotToAxis ? c_rterms_rb_rot
                                               : c_rterms_std;
  const int nt = transfer == kStandard ? 9 : 5;
  T s = Arith<T>::mul(T(rt[0].w), d[sidx(Lf, fi + rt[0].dx, fj + rt[0].dy)]);
  for (int k = 1; k < nt; ++k) s = madd<T, EXACT>(s, T(rt[k].w), d[sidx(Lf, fi + rt[k].dx, fj + rt[k].dy)]);
  fc[sidx(Lc, i, j)] = s;
}

template <typename T, bool EXACT>
__global__ void k_prolong_add(const LevelDev<T>* __restrict__ Lfp, const LevelDev<T>* __restrict__ Lcp,
                              int transfer, T* __restrict__ uf, const T* __restrict__ vc) {
  const LevelDev<T>& Lf = *Lfp;
  const LevelDev<T>& Lc = *Lcp;
  int i, j;
  if (!thread_node(Lf, i, j) || !interior(Lf, i, j)) return;
  const int64_t at = sidx(Lf, i, j);
  T e;
  if (transfer == kRbAxisToRot) {
    if (((i + j) & 1) == 0) {
      e = vc[sidx(Lc, i, j)];
    } else {
      const T q = T(0.25);
      e = Arith<T>::mul(q, vc[sidx(Lc, i, j - 1)]);
      e = madd<T, EXACT>(e, q, vc[sidx(Lc, i - 1, j)]);
      e = madd<T, EXACT>(e, q, vc[sidx(Lc, i + 1, j)]);
      e = madd<T, EXACT>(e, q, vc[sidx(Lc, i, j + 1)]);
    }
  } else if (transfer == kRbRotToAxis) {
    if ((i & 1) == 0) {
      e = vc[sidx(Lc, i >> 1, j >> 1)];
    } else {
      const T q = T(0.25);
      const int i0 = (i - 1) >> 1, i1 = (i + 1) >> 1, j0 = (j - 1) >> 1, j1 = (j + 1) >> 1;
      e = Arith<T>::mul(q, vc[sidx(Lc, i0, j0)]);
      e = madd<T, EXACT>(e, q, vc[sidx(Lc, i1, j0)]);
      e = madd<T, EXACT>(e, q, vc[sidx(Lc, i0, j1)]);
      e = madd<T, EXACT>(e, q, vc[sidx(Lc, i1, j1)]);
    }
  } else {
    int xs[2], ys[2];
    T wx, wy;
    int nx, ny;
    if (i & 1) { xs[0] = (i - 1) >> 1; xs[1] = (i + 1) >> 1; nx = 2; wx = T(0.5); }
    else { xs[0] = i >> 1; nx = 1; wx = T(1); }
    if (j & 1) { ys[0] = (j - 1) >> 1; ys[1] = (j + 1) >> 1; ny = 2; wy = T(0.5); }
    else { ys[0] = j >> 1; ny = 1; wy = T(1); }
    const T w = Arith<T>::mul(wx, wy);  // exact
    bool first = true;
    e = T(0);
    for (int b = 0; b < ny; ++b)
      for (int a = 0; a < nx; ++a) {
        const T x = vc[sidx(Lc, xs[a], ys[b])];
        e = first ? Arith<T>::mul(w, x) : madd<T, EXACT>(e, w, x);
        first = false;
      }
  }
  uf[at] = Arith<T>::add(uf[at], e);
}

template <typename T>
__global__ void k_coarsest(int64_t idx, T a, const T* __restrict__ f, T* __restrict__ u) {
  if (threadIdx.x == 0 && blockIdx.x == 0) u[idx] = Arith<T>::div(f[idx], a);
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

template <typename T, bool EXACT>
__global__ void k_resnorm_partial(const LevelDev<T>* __restrict__ Lp, const T* __restrict__ u,
                                  const T* __restrict__ f, double* __restrict__ partial) {
  const LevelDev<T>& L = *Lp;
  int i, j;
  double v = 0.0;
  if (thread_node(L, i, j) && interior(L, i, j)) {
    const int64_t at = sidx(L, i, j);
    const double d = (double)Arith<T>::sub(f[at], apply_at<T, EXACT>(L, u, i, j, at, nullptr));
    v = d * d;
  }
  v = block_sum(v);
  if (threadIdx.x == 0 && threadIdx.y == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = v;
}

template <typename T>
__global__ void k_sumsq_partial(const LevelDev<T>* __restrict__ Lp, const T* __restrict__ f,
                                double* __restrict__ partial) {
  const LevelDev<T>& L = *Lp;
  int i, j;
  double v = 0.0;
  if (thread_node(L, i, j) && interior(L, i, j)) {
    const double x = (double)f[sidx(L, i, j)];
    v = x * x;
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
template <bool EXACT>
__global__ void k_ir_residual(const LevelDev<double>* __restrict__ Lp, const double* __restrict__ u,
                              const double* __restrict__ f, float* __restrict__ r32, double scale,
                              double* __restrict__ partial) {
  const LevelDev<double>& L = *Lp;
  int i, j;
  double v = 0.0;
  if (thread_node(L, i, j) && interior(L, i, j)) {
    const int64_t at = sidx(L, i, j);
    const double r = Arith<double>::sub(f[at], apply_at<double, EXACT>(L, u, i, j, at, nullptr));
    r32[at] = (float)(r * scale);
    v = r * r;
  }
  v = block_sum(v);
  if (threadIdx.x == 0 && threadIdx.y == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = v;
}

// u += e * inv_scale (FP64 update of the refinement step).
__global__ void k_ir_update(const LevelDev<double>* __restrict__ Lp, double* __restrict__ u,
                            const float* __restrict__ e, double inv_scale) {
  const LevelDev<double>& L = *Lp;
  int i, j;
  if (!thread_node(L, i, j) || !interior(L, i, j)) return;
  const int64_t at = sidx(L, i, j);
  u[at] = u[at] + (double)e[at] * inv_scale;
}

template <typename T>
dim3 grid_of(const LevelDev<T>& L) {
  return dim3((L.cols + kBX - 1) / kBX, (L.rows + kBY - 1) / kBY);
}

}  // namespace

template <typename T>
cudaError_t launch_half_sweep(const LevelPair<T>& L, bool exact, const T* uin, const T* f, T* uout,
                              int red, cudaStream_t s) {
  if (exact) k_half_sweep<T, true><<<grid_of(L.h), dim3(kBX, kBY), 0, s>>>(L.d, uin, f, uout, red);
  else k_half_sweep<T, false><<<grid_of(L.h), dim3(kBX, kBY), 0, s>>>(L.d, uin, f, uout, red);
  return cudaGetLastError();
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

template <typename T>
cudaError_t launch_residual(const LevelPair<T>& L, bool exact, const T* u, const T* f, T* d,
                            cudaStream_t s) {
  if (exact) k_residual<T, true><<<grid_of(L.h), dim3(kBX, kBY), 0, s>>>(L.d, u, f, d);
  else k_residual<T, false><<<grid_of(L.h), dim3(kBX, kBY), 0, s>>>(L.d, u, f, d);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restrict(const LevelPair<T>& Lf, const LevelPair<T>& Lc, int transfer, bool exact,
                            const T* d, T* fc, cudaStream_t s) {
  if (exact) k_restrict<T, true><<<grid_of(Lc.h), dim3(kBX, kBY), 0, s>>>(Lf.d, Lc.d, transfer, d, fc);
  else k_restrict<T, false><<<grid_of(Lc.h), dim3(kBX, kBY), 0, s>>>(Lf.d, Lc.d, transfer, d, fc);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong_add(const LevelPair<T>& Lf, const LevelPair<T>& Lc, int transfer,
                               bool exact, T* uf, const T* vc, cudaStream_t s) {
  if (exact) k_prolong_add<T, true><<<grid_of(Lf.h), dim3(kBX, kBY), 0, s>>>(Lf.d, Lc.d, transfer, uf, vc);
  else k_prolong_add<T, false><<<grid_of(Lf.h), dim3(kBX, kBY), 0, s>>>(Lf.d, Lc.d, transfer, uf, vc);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarsest(int64_t idx, T a, const T* f, T* u, cudaStream_t s) {
  k_coarsest<T><<<1, 32, 0, s>>>(idx, a, f, u);
  return cudaGetLastError();
}

template <typename T>
int resnorm_blocks(const LevelPair<T>& L) {
  const dim3 g = grid_of(L.h);
  return (int)(g.x * g.y);
}

template <typename T>
cudaError_t launch_resnorm(const LevelPair<T>& L, bool exact, const T* u, const T* f,
                           double* partial, double* out, cudaStream_t s) {
  const dim3 g = grid_of(L.h);
  if (exact) k_resnorm_partial<T, true><<<g, dim3(kBX, kBY), 0, s>>>(L.d, u, f, partial);
  else k_resnorm_partial<T, false><<<g, dim3(kBX, kBY), 0, s>>>(L.d, u, f, partial);
  k_sum_partials<<<1, dim3(kBX, kBY), 0, s>>>(partial, (int)(g.x * g.y), out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sumsq(const LevelPair<T>& L, const T* f, double* partial, double* out,
                         cudaStream_t s) {
  const dim3 g = grid_of(L.h);
  k_sumsq_partial<T><<<g, dim3(kBX, kBY), 0, s>>>(L.d, f, partial);
  k_sum_partials<<<1, dim3(kBX, kBY), 0, s>>>(partial, (int)(g.x * g.y), out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_zero_boundary(const LevelPair<T>& L, T* u, cudaStream_t s) {
  const int n = L.h.n;
  k_zero_boundary<T><<<(n + 1 + 255) / 256, 256, 0, s>>>(n, L.h.pitch, u);
  return cudaGetLastError();
}

cudaError_t launch_ir_residual(const LevelPair<double>& L, bool exact, const double* u, const double* f,
                               float* r32, double scale, double* partial, double* out, cudaStream_t s) {
  const dim3 g = grid_of(L.h);
  if (exact) k_ir_residual<true><<<g, dim3(kBX, kBY), 0, s>>>(L.d, u, f, r32, scale, partial);
  else k_ir_residual<false><<<g, dim3(kBX, kBY), 0, s>>>(L.d, u, f, r32, scale, partial);
  k_sum_partials<<<1, dim3(kBX, kBY), 0, s>>>(partial, (int)(g.x * g.y), out);
  return cudaGetLastError();
}

cudaError_t launch_ir_update(const LevelPair<double>& L, double* u, const float* e, double inv_scale,
                             cudaStream_t s) {
  k_ir_update<<<grid_of(L.h), dim3(kBX, kBY), 0, s>>>(L.d, u, e, inv_scale);
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
                                          const T*, T*, cudaStream_t);                                \
  template cudaError_t launch_prolong_add<T>(const LevelPair<T>&, const LevelPair<T>&, int, bool, T*, \
                                             const T*, cudaStream_t);                                 \
  template cudaError_t launch_coarsest<T>(int64_t, T, const T*, T*, cudaStream_t);                    \
  template int resnorm_blocks<T>(const LevelPair<T>&);                                                \
  template cudaError_t launch_resnorm<T>(const LevelPair<T>&, bool, const T*, const T*, double*,     \
                                         double*, cudaStream_t);                                      \
  template cudaError_t launch_sumsq<T>(const LevelPair<T>&, const T*, double*, double*, cudaStream_t); \
  template cudaError_t launch_zero_boundary<T>(const LevelPair<T>&, T*, cudaStream_t);

NSMG_INSTANTIATE(double)
NSMG_INSTANTIATE(float)

}  // namespace nsmg

// ---------------------------------------------------------------------------
// Relative residual of the finest level without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// residual norm: code running while a CUDA stream is being captured into a graph
// (cudaMalloc is not capturable), real-time loops that must not hit the implicit
// device synchronisation of cudaMalloc / cudaFree, or hosts that hand the library a
// fixed memory budget and forbid allocation after set-up. For them the partial sums
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
