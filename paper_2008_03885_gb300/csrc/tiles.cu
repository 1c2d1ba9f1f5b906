// Shared-memory tile kernels for the large axis levels of the FP32 inner cycle (see
// tiles.h). A block owns a tile of kTQ storage columns x kTJ rows (kTQ / 2 node pairs
// per row, each pair one red and one black node). One TMA load per input array brings
// the tile and its halo into shared memory (zero fill outside the array); the block then
// runs its relaxation phases on shared-memory copies, recomputing on the halo what the
// next phase needs (red nodes of one phase on a margin of the stencil reach around the
// nodes the following phase updates), and writes only the tile's result. Values of one
// colour are kept compactly, one per node pair, so that consecutive lanes touch
// consecutive shared-memory words.
//
// Arithmetic per node is exactly that of the per-step kernels (kernels.cu): the same
// fast stencil in registers (a 5-point or 9-point cross, terms in evaluation order) or
// the same boundary-class term list, the same grouped sums (or fused multiply-adds), and
// the same relaxation u + r * omega / a_pp; so a fused group of steps gives the same bits
// as the separate launches.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <type_traits>
#include <utility>

#include "device.cuh"
#include "tiles.h"

namespace nsmg {
namespace {

constexpr int kTQ = 128;  // tile storage columns
constexpr int kTP = kTQ / 2;  // node pairs per tile row
constexpr int kTJ = 32;   // tile rows
constexpr int kTT = 256;  // threads per block
constexpr int kTileMinRows = 256;  // smaller levels keep the per-step kernels

__host__ __device__ constexpr int round4(int x) { return (x + 3) / 4 * 4; }

// A compact one-colour array over the tile plus a margin of M rows and MP node pairs.
template <int M>
struct Reg {
  static constexpr int mp = (M + 1) / 2;
  static constexpr int w = kTP + 2 * mp;
  static constexpr int h = kTJ + 2 * M;
  static constexpr int n = w * h;
};

// Halo of the TMA box (x multiple of 4 elements: the box must start on 16 bytes).
template <int R, int NS>
struct PreGeo {  // presmooth: red(0) values on the tile plus (2 NS - 1) R
  static constexpr int M0 = (2 * NS - 1) * R;
  static constexpr int HX = round4(2 * Reg<M0>::mp), HY = M0;
};
template <int R>
struct SweepGeo {  // one sweep: red on the tile plus R, reading u a further R away
  static constexpr int HX = round4(2 * Reg<R>::mp + R), HY = 2 * R;
};
template <int R>
struct RrGeo {  // residual + restriction: red residuals on the tile plus 1
  static constexpr int HX = round4(2 * Reg<1>::mp + R), HY = 1 + R;
};

// ---- mbarrier and TMA --------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load(float* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bound of the waits on a load barrier (each try_wait suspends the thread for a short
// system-dependent time; the limit is far beyond any real load).
constexpr long kWaitTries = 1L << 22;

// ---- node arithmetic -------------------------------------------------------------
// omega / a_pp of node (i, j).
__device__ __forceinline__ float wd_at(const LevelDev<float>& L, float wdf, int i, int j) {
  return fast_node_c<false>(L, i, j) ? wdf : L.cls_wd[class_of(L, i, j)];
}

// Relaxed value u + (f - s) omega / a_pp (as relax_fast / relax_value).
template <bool EXACT>
__device__ __forceinline__ float relax(float s, float f, float u, float wd) {
  const float r = Arith<float>::sub(f, s);
  return EXACT ? Arith<float>::add(u, Arith<float>::mul(r, wd)) : Arith<float>::fma(r, wd, u);
}

// The wide stencils of the second and third red-black Galerkin axis levels (Eq. L_G_l
// from the 5-point operator; Sec. 4.4) in evaluation order. 21 points (reach 2): its
// groups of equal coefficient are the eight (1, 2) knight neighbours, the four (2, 0)
// neighbours, the four diagonal and the four (1, 0) neighbours, the centre. 37 points
// (reach 3): the eight (1, 3), the four (3, 0), the four (2, 2), the eight (1, 2), the
// four (2, 0), the four diagonal and the four (1, 0) neighbours, the centre. Each group
// in (dy, dx) order; gstart marks a group's first term.
template <int NT>
__host__ __device__ constexpr int wide_dx(int k) {
  if constexpr (NT == 21) {
    constexpr int x[21] = {-1, 1, -2, 2, -2, 2, -1, 1, 0, -2, 2, 0, -1, 1, -1, 1, 0, -1, 1, 0, 0};
    return x[k];
  } else {
    constexpr int x[37] = {-1, 1, -3, 3, -3, 3, -1, 1, 0, -3, 3, 0, -2, 2, -2, 2, -1, 1, -2,
                           2,  -2, 2, -1, 1, 0, -2, 2, 0, -1, 1, -1, 1, 0, -1, 1, 0, 0};
    return x[k];
  }
}
template <int NT>
__host__ __device__ constexpr int wide_dy(int k) {
  if constexpr (NT == 21) {
    constexpr int y[21] = {-2, -2, -1, -1, 1, 1, 2, 2, -2, 0, 0, 2, -1, -1, 1, 1, -1, 0, 0, 1, 0};
    return y[k];
  } else {
    constexpr int y[37] = {-3, -3, -1, -1, 1, 1, 3, 3, -3, 0, 0, 3, -2, -2, 2, 2, -2, -2, -1,
                           -1, 1,  1,  2,  2, -2, 0, 0, 2, -1, -1, 1, 1, -1, 0, 0, 1, 0};
    return y[k];
  }
}
template <int NT>
__host__ __device__ constexpr bool wide_gstart(int k) {
  if constexpr (NT == 21) return k == 0 || k == 8 || k == 12 || k == 16 || k == 20;
  else return k == 0 || k == 8 || k == 12 || k == 16 || k == 24 || k == 28 || k == 32 || k == 36;
}
__host__ __device__ constexpr bool wide_nt(int nt) { return nt == 21 || nt == 37; }
// stencil reach of the NT-term fast stencils of the axis tile kernels
__host__ __device__ constexpr int tile_reach(int nt) { return nt == 5 ? 1 : nt == 37 ? 3 : 2; }

// (L x)(i, j) at a node outside the fast range: its boundary-class term list.
template <bool EXACT, class X>
__device__ __forceinline__ float class_stencil(const LevelDev<float>& L, int i, int j, X x) {
  const int2 e = L.cls[class_of(L, i, j)];
  const ClassTerm<float>* tt = L.terms + e.x;
  RowSum<float, EXACT> acc;
#pragma unroll 4
  for (int k = 0; k < e.y; ++k) {
    const Term<float> t = load_term(tt + k);
    acc.add(t.c, x(i + t.dx, j + t.dy), t.start);
  }
  return acc.value();
}

// (L x)(i, j): the fast cross stencil with coefficients c (in evaluation order) or the
// node's boundary-class term list. x(i, j) returns the value of lattice node (i, j).
template <bool EXACT, int NT, class X>
__device__ __forceinline__ float stencil(const LevelDev<float>& L, const float (&c)[NT], int i, int j, X x) {
  if (fast_node_c<false>(L, i, j)) {
    // terms in evaluation order: 9 points = +-2 neighbours, +-1 neighbours, centre;
    // 5 points = the four neighbours, the centre; 21 and 37 points as wide_dx / wide_dy
    RowSum<float, EXACT> acc;
    if constexpr (wide_nt(NT)) {
#pragma unroll
      for (int k = 0; k < NT; ++k) acc.add(c[k], x(i + wide_dx<NT>(k), j + wide_dy<NT>(k)), wide_gstart<NT>(k));
    } else if (NT == 9) {
      acc.add(c[0], x(i, j - 2), true);
      acc.add(c[1], x(i - 2, j), false);
      acc.add(c[2], x(i + 2, j), false);
      acc.add(c[3], x(i, j + 2), false);
      acc.add(c[4], x(i, j - 1), true);
      acc.add(c[5], x(i - 1, j), false);
      acc.add(c[6], x(i + 1, j), false);
      acc.add(c[7], x(i, j + 1), false);
      acc.add(c[8], x(i, j), true);
    } else {
      acc.add(c[0], x(i, j - 1), true);
      acc.add(c[1], x(i - 1, j), false);
      acc.add(c[2], x(i + 1, j), false);
      acc.add(c[3], x(i, j + 1), false);
      acc.add(c[4], x(i, j), true);
    }
    return acc.value();
  }
  return class_stencil<EXACT>(L, i, j, x);
}

// Tile origin of the block.
struct Tile {
  int J0, Q0, P0;
  __device__ Tile(int bx, int by) : J0(by * kTJ), Q0(bx * kTQ), P0(bx * kTP) {}
  // index of lattice node (i, j) in a compact one-colour array of margin M
  template <int M>
  __device__ __forceinline__ int at(int i, int j) const {
    return (j - J0 + M) * Reg<M>::w + ((i >> 1) - P0 + Reg<M>::mp);
  }
  // index of lattice node (i, j) in a staged box with halo (HX, HY)
  template <int HX, int HY>
  __device__ __forceinline__ int box(int i, int j) const {
    return (j - J0 + HY) * (kTQ + 2 * HX) + (i - Q0 + HX);
  }
};

__device__ __forceinline__ bool inner(int n, int i, int j) { return i >= 1 && i < n && j >= 1 && j < n; }

// TMA destinations start on 128-byte boundaries: the dynamic shared memory is rounded
// up to one (the launch adds 128 bytes for it) and every staged box is padded to a
// multiple of 32 floats.
__host__ __device__ constexpr int pad32(int n) { return (n + 31) / 32 * 32; }
__device__ __forceinline__ float* smem_base(unsigned char* raw) {
  return reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(raw) + 127) & ~(uintptr_t)127);
}

// Store the tile's result: node pair (2p, 2p + 1) of row j as one 8-byte store.
__device__ __forceinline__ void store_pair(float* out, int pitch, int n, int j, int p, float red, float black) {
  if (j > n || 2 * p > n) return;
  const float2 v = (j & 1) ? make_float2(red, black) : make_float2(black, red);  // red: i + j odd
  *reinterpret_cast<float2*>(out + (int64_t)j * pitch + 2 * p) = v;
}

// ---- fast path: tiles whose nodes (with the halo) are all fast interior nodes ------
// Then every node uses the level's cross stencil with the coefficients in registers,
// omega / a_pp is the level's constant, and no node needs a boundary test: each value
// is read at a compile-time offset from a per-node base index. A source is where a
// phase reads one colour (or both) from:
struct SZero {  // the zero start: every value of this colour is 0
  template <int M>
  __device__ __forceinline__ int base(int, int, int) const { return 0; }
  template <int DX, int DY>
  __device__ __forceinline__ float get(int, int) const { return 0.f; }
};
template <int MS>
struct SCompact {  // one colour, one value per node pair, tile plus margin MS
  const float* p;
  // base of the node at (row rr, pair pp) of a region of margin M
  template <int M>
  __device__ __forceinline__ int base(int rr, int pp, int) const {
    return (rr - M + MS) * Reg<MS>::w + (pp - Reg<M>::mp + Reg<MS>::mp);
  }
  // lattice offset (DX, DY) from a node whose column parity within its pair is a
  template <int DX, int DY>
  __device__ __forceinline__ float get(int b, int a) const {
    return p[b + DY * Reg<MS>::w + ((a + DX) >> 1)];
  }
};
template <int HX, int HY>
struct SBox {  // a staged TMA box (both colours), halo (HX, HY)
  const float* p;
  static constexpr int BW = kTQ + 2 * HX;
  template <int M>
  __device__ __forceinline__ int base(int rr, int pp, int a) const {
    return (rr - M + HY) * BW + (2 * (pp - Reg<M>::mp) + a + HX);
  }
  template <int DX, int DY>
  __device__ __forceinline__ float get(int b, int) const {
    return p[b + DY * BW + DX];
  }
};

// Term K of a wide stencil: odd offsets read the other colour's source.
template <int NT, int K, class SO, class SS>
__device__ __forceinline__ float term_wide(const SO& so, int bo, const SS& ss, int bs, int a) {
  constexpr int DX = wide_dx<NT>(K), DY = wide_dy<NT>(K);
  if constexpr (((DX + DY) & 1) != 0) return so.template get<DX, DY>(bo, a);
  else return ss.template get<DX, DY>(bs, a);
}
template <bool EXACT, int NT, class SO, class SS, int... K>
__device__ __forceinline__ float cross_wide(const float (&c)[NT], const SO& so, int bo, const SS& ss, int bs, int a,
                                           std::integer_sequence<int, K...>) {
  const float x[NT] = {term_wide<NT, K>(so, bo, ss, bs, a)...};
  if constexpr (EXACT) {
    RowSum<float, true> acc;
#pragma unroll
    for (int k = 0; k < NT; ++k) acc.add(c[k], x[k], wide_gstart<NT>(k));
    return acc.value();
  } else {
    float s = Arith<float>::mul(c[0], x[0]);
#pragma unroll
    for (int k = 1; k < NT; ++k) s = Arith<float>::fma(c[k], x[k], s);
    return s;
  }
}

// (L x) at a fast node: terms in (dy, dx) order; odd offsets (DX + DY) read the other
// colour's source `so` (base bo), even ones the node's own colour `ss` (base bs).
template <bool EXACT, int NT, class SO, class SS>
__device__ __forceinline__ float cross(const float (&c)[NT], const SO& so, int bo, const SS& ss, int bs, int a) {
  // terms in evaluation order (group-major, see LevelDev::c): 9 points = the four
  // +-2 neighbours, the four +-1 neighbours, the centre; 5 points = the four neighbours,
  // the centre; 21 and 37 points: see wide_dx
  if constexpr (wide_nt(NT)) {
    return cross_wide<EXACT, NT>(c, so, bo, ss, bs, a, std::make_integer_sequence<int, NT>{});
  } else if constexpr (NT == 9) {
    const float x0 = ss.template get<0, -2>(bs, a), x1 = ss.template get<-2, 0>(bs, a);
    const float x2 = ss.template get<2, 0>(bs, a), x3 = ss.template get<0, 2>(bs, a);
    const float x4 = so.template get<0, -1>(bo, a), x5 = so.template get<-1, 0>(bo, a);
    const float x6 = so.template get<1, 0>(bo, a), x7 = so.template get<0, 1>(bo, a);
    const float x8 = ss.template get<0, 0>(bs, a);
    if constexpr (EXACT) {
      const float g0 = Arith<float>::add(Arith<float>::add(Arith<float>::add(x0, x1), x2), x3);
      const float g1 = Arith<float>::add(Arith<float>::add(Arith<float>::add(x4, x5), x6), x7);
      return Arith<float>::add(Arith<float>::add(Arith<float>::mul(c[0], g0), Arith<float>::mul(c[4], g1)),
                               Arith<float>::mul(c[8], x8));
    } else {
      float s = Arith<float>::mul(c[0], x0);
      s = Arith<float>::fma(c[1], x1, s);
      s = Arith<float>::fma(c[2], x2, s);
      s = Arith<float>::fma(c[3], x3, s);
      s = Arith<float>::fma(c[4], x4, s);
      s = Arith<float>::fma(c[5], x5, s);
      s = Arith<float>::fma(c[6], x6, s);
      s = Arith<float>::fma(c[7], x7, s);
      return Arith<float>::fma(c[8], x8, s);
    }
  } else {
    const float x0 = so.template get<0, -1>(bo, a), x1 = so.template get<-1, 0>(bo, a);
    const float x2 = so.template get<1, 0>(bo, a), x3 = so.template get<0, 1>(bo, a);
    const float x4 = ss.template get<0, 0>(bs, a);
    if constexpr (EXACT) {
      const float g0 = Arith<float>::add(Arith<float>::add(Arith<float>::add(x0, x1), x2), x3);
      return Arith<float>::add(Arith<float>::mul(c[0], g0), Arith<float>::mul(c[4], x4));
    } else {
      float s = Arith<float>::mul(c[0], x0);
      s = Arith<float>::fma(c[1], x1, s);
      s = Arith<float>::fma(c[2], x2, s);
      s = Arith<float>::fma(c[3], x3, s);
      return Arith<float>::fma(c[4], x4, s);
    }
  }
}

// Fast value of element (rr, pp) (column parity a) of a relaxation phase of margin M:
// relax(L x, f, old) (old, so and ss as above; with ZERO_START the stencil-free value
// 0 + f omega / a_pp).
template <bool EXACT, int NT, int M, bool ZERO_START, class SO, class SS, class SOLD, class FB>
__device__ __forceinline__ float fast_value(const float (&c)[NT], float wd, const SO& so, const SS& ss,
                                            const SOLD& sold, const FB& fb, int rr, int pp, int a) {
  const float f = fb.template get<0, 0>(fb.template base<M>(rr, pp, a), a);
  if constexpr (ZERO_START) {
    return relax_from_zero(f, wd);
  } else {
    const float st = cross<EXACT, NT>(c, so, so.template base<M>(rr, pp, a), ss, ss.template base<M>(rr, pp, a), a);
    return relax<EXACT>(st, f, sold.template get<0, 0>(sold.template base<M>(rr, pp, a), a), wd);
  }
}

// One fast relaxation phase: every node of colour RED in the tile plus margin M gets its
// fast value, handed to sink(e, rr, pp, a, value) (e = rr * w + pp).
// (Measured on GB300, 4097^2 FP32 fourth order, one tile per block: 2 and 4 nodes per
// thread at a time were slower than 1 -- presmooth 107 / 134 vs 106 us, sweep 70 / 86 vs
// 67 us -- with more registers per node and more idle lanes in each phase's last pass.)
template <bool EXACT, int NT, bool RED, int M, bool ZERO_START, class SO, class SS, class SOLD, class FB, class SINK>
__device__ __forceinline__ void phase(const float (&c)[NT], float wd, const SO& so, const SS& ss, const SOLD& sold,
                                      const FB& fb, SINK sink) {
  for (int e = threadIdx.x; e < Reg<M>::n; e += kTT) {
    const int rr = e / Reg<M>::w, pp = e - rr * Reg<M>::w;
    const int a = (rr + M + (RED ? 1 : 0)) & 1;  // column parity of the node (tile rows start even)
    sink(e, rr, pp, a, fast_value<EXACT, NT, M, ZERO_START>(c, wd, so, ss, sold, fb, rr, pp, a));
  }
}

// Lattice coordinates of element (rr, pp) (column parity a) of a region of margin M.
template <int M>
__device__ __forceinline__ void node_of(const Tile& T, int rr, int pp, int a, int& i, int& j) {
  j = T.J0 - M + rr;
  i = 2 * (T.P0 - Reg<M>::mp + pp) + a;
}

// Strips of a region of margin M (tile T of level L) that hold its nodes outside the
// fast range (rx <= i <= fxe, ry <= j <= fye) within rows 0 <= j <= n and columns
// 0 <= i <= n + 1: rows [r0, rt) and [rb, r1), and in the rows between them the pairs
// [p0, pl) and [pr, p1). A superset of those nodes, without overlap. Nodes beyond those
// rows and columns are never read (fast stencils stay two nodes inside the boundary,
// boundary-class rows drop boundary columns) nor stored, so they are left unset.
template <int M>
struct Strips {
  int r0, rt, rb, r1, p0, pl, pr, p1, pw, mw, count;
  __device__ __forceinline__ Strips(const LevelDev<float>& L, const Tile& T) {
    constexpr int W = Reg<M>::w, H = Reg<M>::h;
    const int j0 = T.J0 - M, q0 = T.P0 - Reg<M>::mp;  // lattice row / pair index of element (0, 0)
    r0 = min(max(-j0, 0), H);
    r1 = max(r0, min(L.n + 1 - j0, H));
    rt = min(max(L.ry - j0, r0), r1);
    rb = max(rt, min(max(L.fye + 1 - j0, r0), r1));
    p0 = min(max(-q0, 0), W);
    p1 = max(p0, min((L.n + 1) / 2 + 1 - q0, W));      // pairs q <= (n + 1) / 2
    pl = min(max(L.rx / 2 + 1 - q0, p0), p1);           // pair q holds i = 2q + a < rx only if q <= rx / 2
    pr = max(pl, min(max(L.fxe / 2 - q0, p0), p1));    // ... i > fxe only if q >= fxe / 2
    pw = p1 - p0;
    mw = (pl - p0) + (p1 - pr);
    count = (rt - r0 + r1 - rb) * pw + (rb - rt) * mw;
  }
  // element k of the strips
  __device__ __forceinline__ void at(int k, int& rr, int& pp) const {
    const int k1 = (rt - r0) * pw, k2 = k1 + (r1 - rb) * pw;
    if (k < k1) {
      const int q = k / pw;
      rr = r0 + q;
      pp = p0 + (k - q * pw);
    } else if (k < k2) {
      const int q = (k - k1) / pw;
      rr = rb + q;
      pp = p0 + (k - k1 - q * pw);
    } else {
      const int q = (k - k2) / mw, r = k - k2 - q * mw;
      rr = rt + q;
      pp = r < pl - p0 ? p0 + r : pr + (r - (pl - p0));
    }
  }
};

// Rows [fast_row0, fast_row0 + fast_rows) of a region of margin M: those that hold
// nodes of the fast range (ry <= j <= fye).
template <int M>
__device__ __forceinline__ int fast_row0(const LevelDev<float>& L, const Tile& T) {
  return min(max(L.ry - (T.J0 - M), 0), Reg<M>::h);
}
template <int M>
__device__ __forceinline__ int fast_rows(const LevelDev<float>& L, const Tile& T, int r0) {
  return max(min(L.fye + 1 - (T.J0 - M), Reg<M>::h) - r0, 0);
}

// The same phase in a tile that reaches the level's boundary strip: the nodes of the
// fast range get their fast value; every other node of the region (a boundary-class
// node, or a node off the interior) gets gen(i, j), the value the per-step kernels give
// it (class terms, omega / a_pp of its class; 0 or the old value off the interior).
// The second pass walks only the strips, so that those nodes share warps.
template <bool EXACT, int NT, bool RED, int M, bool ZERO_START, class SO, class SS, class SOLD, class FB, class SINK,
          class GEN>
__device__ __forceinline__ void phase_edge(const float (&c)[NT], float wd, const SO& so, const SS& ss,
                                           const SOLD& sold, const FB& fb, SINK sink, const LevelDev<float>& L,
                                           const Tile& T, GEN gen) {
  const int fr0 = fast_row0<M>(L, T), nf = fast_rows<M>(L, T, fr0) * Reg<M>::w;
  for (int e = threadIdx.x; e < nf; e += kTT) {
    const int rq = e / Reg<M>::w, pp = e - rq * Reg<M>::w, rr = fr0 + rq;
    const int a = (rr + M + (RED ? 1 : 0)) & 1;
    int i, j;
    node_of<M>(T, rr, pp, a, i, j);
    if (!fast_node_c<false>(L, i, j)) continue;
    sink(rr * Reg<M>::w + pp, rr, pp, a, fast_value<EXACT, NT, M, ZERO_START>(c, wd, so, ss, sold, fb, rr, pp, a));
  }
  const Strips<M> st(L, T);
  for (int k = threadIdx.x; k < st.count; k += kTT) {
    int rr, pp;
    st.at(k, rr, pp);
    const int a = (rr + M + (RED ? 1 : 0)) & 1;
    int i, j;
    node_of<M>(T, rr, pp, a, i, j);
    if (fast_node_c<false>(L, i, j)) continue;
    sink(rr * Reg<M>::w + pp, rr, pp, a, gen(i, j));
  }
}

// Whether the tile's nodes within margin m (rows) / 2 mp (columns) are all fast
// interior nodes of L (Dirichlet levels: rx <= i <= n - rx, ry <= j <= n - ry).
template <int M>
__device__ __forceinline__ bool fast_tile(const LevelDev<float>& L, const Tile& T) {
  return T.Q0 - 2 * Reg<M>::mp >= L.rx && T.Q0 + kTQ + 2 * Reg<M>::mp - 1 <= L.fxe && T.J0 - M >= L.ry &&
         T.J0 + kTJ - 1 + M <= L.fye;
}

// Unchecked store of a fast tile's node pair (2p, 2p + 1) of row j.
__device__ __forceinline__ void put_pair(float* out, int pitch, int j, int p, float red, float black) {
  const float2 v = (j & 1) ? make_float2(red, black) : make_float2(black, red);
  *reinterpret_cast<float2*>(out + (int64_t)j * pitch + 2 * p) = v;
}

// ---- one tile per block ---------------------------------------------------------
// Block (bx, by) stages its tile with one TMA load per input array and runs body(T,
// box) on it. (Measured on GB300, 4097^2 FP32 fourth order: a persistent form with two
// shared-memory stages, the next tile's loads in flight during the current one, was
// slower: sweep 78 vs 67 us, presmooth 126 vs 106 us; it holds two blocks per SM
// instead of three.) A wait that gives up sets the status word and leaves the block
// once its load has landed (or a second bounded wait ran out).
__device__ __forceinline__ bool wait_tile(uint64_t* bar, int* status) {
  bool ok = false;
  for (long q = 0; q < kWaitTries && !ok; ++q) ok = mbar_try(bar, 0);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) {
      atomicOr(status, kStatusTmaTimeout);
      for (long q = 0; q < kWaitTries && !mbar_try(bar, 0); ++q) {
      }
    }
    __syncthreads();
    return false;
  }
  return true;
}

template <int NB, class BODY>
__device__ __forceinline__ void tile_block(float* box0, int box_floats, const CUtensorMap* const (&maps)[NB], int hx,
                                           int hy, int* status, BODY body) {
  __shared__ uint64_t bar;
  const Tile T(blockIdx.x, blockIdx.y);
  if (threadIdx.x == 0) {
    mbar_init(&bar);
    mbar_expect(&bar, (uint32_t)(NB * (kTQ + 2 * hx) * (kTJ + 2 * hy) * sizeof(float)));
#pragma unroll
    for (int m = 0; m < NB; ++m) tma_load(box0 + m * box_floats, maps[m], T.Q0 - hx, T.J0 - hy, &bar);
  }
  __syncthreads();
  if (!wait_tile(&bar, status)) return;
  body(T, box0);
}

// ---- presmooth: NS red-black sweeps from u = 0 ---------------------------------
template <bool EXACT, int NT, int NS>
__global__ void __launch_bounds__(kTT, 3) k_tile_presmooth(const LevelDev<float>* __restrict__ Lp,
                                                        const __grid_constant__ CUtensorMap mapF,
                                                        float* __restrict__ out, int* __restrict__ status) {
  constexpr int R = tile_reach(NT);
  using G = PreGeo<R, NS>;
  constexpr int M0 = G::M0, M1 = (2 * NS - 2) * R, M2 = NS == 2 ? R : 0;
  constexpr int FN = (kTQ + 2 * G::HX) * (kTJ + 2 * G::HY);
  extern __shared__ __align__(128) unsigned char tile_smem[];
  float* box0 = smem_base(tile_smem);
  float* sR0 = box0 + pad32(FN);
  float* sB1 = sR0 + Reg<M0>::n;
  float* sR2 = sB1 + (NS == 2 ? Reg<M1>::n : 0);
  const LevelDev<float>& L = *Lp;
  float c[NT];
#pragma unroll
  for (int k = 0; k < NT; ++k) c[k] = L.c[k];
  const float wdf = L.wd;
  const int n = L.n, pitch = L.pitch;
  const CUtensorMap* const maps[1] = {&mapF};
  tile_block<1>(box0, pad32(FN), maps, G::HX, G::HY, status, [&](const Tile& T, float* sF) {
    const SBox<G::HX, G::HY> fb{sF};
    const SCompact<M0> r0{sR0};
    auto F = [=](int i, int j) { return sF[T.box<G::HX, G::HY>(i, j)]; };
    auto xR0 = [=](int i, int j) { return sR0[T.at<M0>(i, j)]; };
    auto xB1 = [=](int i, int j) { return sB1[T.at<M1>(i, j)]; };
    auto xR2 = [=](int i, int j) { return sR2[T.at<M2>(i, j)]; };
    // values of the nodes outside the fast range, phase by phase (as the per-step kernels)
    auto g0 = [=](int i, int j) {  // red from zero: 0 + f omega / a_pp
      return inner(n, i, j) ? relax_from_zero(F(i, j), wd_at(L, wdf, i, j)) : 0.f;
    };
    auto g1 = [=](int i, int j) {  // black of sweep 1 (old values 0)
      if (!inner(n, i, j)) return 0.f;
      const float st = stencil<EXACT, NT>(L, c, i, j, [=](int x, int y) { return ((x + y) & 1) ? xR0(x, y) : 0.f; });
      return relax<EXACT>(st, F(i, j), 0.f, wd_at(L, wdf, i, j));
    };
    auto g2 = [=](int i, int j) {  // red of sweep 2
      if (!inner(n, i, j)) return 0.f;
      const float st =
          stencil<EXACT, NT>(L, c, i, j, [=](int x, int y) { return ((x + y) & 1) ? xR0(x, y) : xB1(x, y); });
      return relax<EXACT>(st, F(i, j), xR0(i, j), wd_at(L, wdf, i, j));
    };
    auto g3 = [=](int i, int j) {  // black of the last sweep, on the tile
      if (!inner(n, i, j)) return 0.f;
      if constexpr (NS == 2) {
        const float st =
            stencil<EXACT, NT>(L, c, i, j, [=](int x, int y) { return ((x + y) & 1) ? xR2(x, y) : xB1(x, y); });
        return relax<EXACT>(st, F(i, j), xB1(i, j), wd_at(L, wdf, i, j));
      } else {
        const float st = stencil<EXACT, NT>(L, c, i, j, [=](int x, int y) { return ((x + y) & 1) ? xR0(x, y) : 0.f; });
        return relax<EXACT>(st, F(i, j), 0.f, wd_at(L, wdf, i, j));
      }
    };
    // a phase over the fast range (every node in a fast tile), else with the others from gen
    auto run = [&](auto check) {
      constexpr bool EDGE = decltype(check)::value;
      auto go = [&](auto red, auto m, auto zero, const auto& so, const auto& ss, const auto& sold, auto sink, auto gen) {
        constexpr bool RED = decltype(red)::value, ZERO = decltype(zero)::value;
        constexpr int MM = decltype(m)::value;
        if constexpr (EDGE) phase_edge<EXACT, NT, RED, MM, ZERO>(c, wdf, so, ss, sold, fb, sink, L, T, gen);
        else phase<EXACT, NT, RED, MM, ZERO>(c, wdf, so, ss, sold, fb, sink);
      };
      using T1 = std::true_type;
      using F0 = std::false_type;
      go(T1{}, std::integral_constant<int, M0>{}, T1{}, SZero{}, SZero{}, SZero{},
         [=](int e, int, int, int, float v) { sR0[e] = v; }, g0);
      __syncthreads();
      // the last phase's result with its red partner, one 8-byte store per node pair
      // (bounds-checked in tiles that reach the level's edge)
      auto put = [=](int rr, int pp, float red, float black) {
        if constexpr (EDGE) store_pair(out, pitch, n, T.J0 + rr, T.P0 + pp, red, black);
        else put_pair(out, pitch, T.J0 + rr, T.P0 + pp, red, black);
      };
      if constexpr (NS == 2) {
        const SCompact<M1> b1{sB1};
        const SCompact<M2> r2{sR2};
        go(F0{}, std::integral_constant<int, M1>{}, F0{}, r0, SZero{}, SZero{},
           [=](int e, int, int, int, float v) { sB1[e] = v; }, g1);
        __syncthreads();
        go(T1{}, std::integral_constant<int, M2>{}, F0{}, b1, r0, r0, [=](int e, int, int, int, float v) { sR2[e] = v; },
           g2);
        __syncthreads();
        go(F0{}, std::integral_constant<int, 0>{}, F0{}, r2, b1, b1,
           [=](int, int rr, int pp, int a, float v) { put(rr, pp, sR2[r2.template base<0>(rr, pp, a)], v); }, g3);
      } else {
        go(F0{}, std::integral_constant<int, 0>{}, F0{}, r0, SZero{}, SZero{},
           [=](int, int rr, int pp, int a, float v) { put(rr, pp, sR0[r0.template base<0>(rr, pp, a)], v); }, g3);
      }
    };
    if (fast_tile<M0>(L, T)) run(std::false_type{});
    else run(std::true_type{});
  });
}

// ---- one red-black sweep, u -> out -----------------------------------------------
template <bool EXACT, int NT>
__global__ void __launch_bounds__(kTT, 3) k_tile_sweep(const LevelDev<float>* __restrict__ Lp,
                                                    const __grid_constant__ CUtensorMap mapU,
                                                    const __grid_constant__ CUtensorMap mapF, float* __restrict__ out,
                                                    int* __restrict__ status) {
  constexpr int R = tile_reach(NT);
  using G = SweepGeo<R>;
  constexpr int BN = (kTQ + 2 * G::HX) * (kTJ + 2 * G::HY);
  extern __shared__ __align__(128) unsigned char tile_smem[];
  float* box0 = smem_base(tile_smem);
  float* sR = box0 + 2 * pad32(BN);
  const LevelDev<float>& L = *Lp;
  float c[NT];
#pragma unroll
  for (int k = 0; k < NT; ++k) c[k] = L.c[k];
  const float wdf = L.wd;
  const int n = L.n, pitch = L.pitch;
  const CUtensorMap* const maps[2] = {&mapU, &mapF};
  tile_block<2>(box0, pad32(BN), maps, G::HX, G::HY, status, [&](const Tile& T, float* sU) {
    float* sF = sU + pad32(BN);
    const SBox<G::HX, G::HY> ub{sU}, fb{sF};
    const SCompact<R> rn{sR};
    auto U = [=](int i, int j) { return sU[T.box<G::HX, G::HY>(i, j)]; };
    auto F = [=](int i, int j) { return sF[T.box<G::HX, G::HY>(i, j)]; };
    auto xR = [=](int i, int j) { return sR[T.at<R>(i, j)]; };
    auto gr = [=](int i, int j) {  // red half-sweep on the tile plus R, nodes outside the fast range
      const float v = U(i, j);
      return inner(n, i, j) ? relax<EXACT>(stencil<EXACT, NT>(L, c, i, j, U), F(i, j), v, wd_at(L, wdf, i, j)) : v;
    };
    auto gb = [=](int i, int j) {  // black half-sweep on the tile, nodes outside the fast range
      const float v = U(i, j);
      if (!inner(n, i, j)) return v;
      const float st = stencil<EXACT, NT>(L, c, i, j, [=](int x, int y) { return ((x + y) & 1) ? xR(x, y) : U(x, y); });
      return relax<EXACT>(st, F(i, j), v, wd_at(L, wdf, i, j));
    };
    auto run = [&](auto check) {
      constexpr bool EDGE = decltype(check)::value;
      auto sink_r = [=](int e, int, int, int, float v) { sR[e] = v; };
      auto sink_b = [=](int, int rr, int pp, int a, float v) {
        const float red = sR[rn.template base<0>(rr, pp, a)];
        if constexpr (EDGE) store_pair(out, pitch, n, T.J0 + rr, T.P0 + pp, red, v);
        else put_pair(out, pitch, T.J0 + rr, T.P0 + pp, red, v);
      };
      if constexpr (EDGE) {
        phase_edge<EXACT, NT, true, R, false>(c, wdf, ub, ub, ub, fb, sink_r, L, T, gr);
        __syncthreads();
        phase_edge<EXACT, NT, false, 0, false>(c, wdf, rn, ub, ub, fb, sink_b, L, T, gb);
      } else {
        phase<EXACT, NT, true, R, false>(c, wdf, ub, ub, ub, fb, sink_r);
        __syncthreads();
        phase<EXACT, NT, false, 0, false>(c, wdf, rn, ub, ub, fb, sink_b);
      }
    };
    if (fast_tile<R>(L, T)) run(std::false_type{});
    else run(std::true_type{});
  });
}

// ---- residual + red-black restriction (axis level -> its black points) ------------
template <bool EXACT, int NT, bool TC>
__global__ void __launch_bounds__(kTT, 3) k_tile_res_restrict(const LevelDev<float>* __restrict__ Lp,
                                                           const LevelDev<float>* __restrict__ Lcp,
                                                           const __grid_constant__ CUtensorMap mapU,
                                                           const __grid_constant__ CUtensorMap mapF,
                                                           float* __restrict__ fc, float* __restrict__ tc,
                                                           int* __restrict__ status) {
  constexpr int R = tile_reach(NT);
  using G = RrGeo<R>;
  constexpr int BN = (kTQ + 2 * G::HX) * (kTJ + 2 * G::HY);
  extern __shared__ __align__(128) unsigned char tile_smem[];
  float* box0 = smem_base(tile_smem);
  float* sD = box0 + 2 * pad32(BN);  // residuals of the red nodes, tile plus 1
  const LevelDev<float>& L = *Lp;
  const LevelDev<float>& Lc = *Lcp;
  float c[NT];
#pragma unroll
  for (int k = 0; k < NT; ++k) c[k] = L.c[k];
  const int n = L.n, pc = Lc.pitch;
  const CUtensorMap* const maps[2] = {&mapU, &mapF};
  tile_block<2>(box0, pad32(BN), maps, G::HX, G::HY, status, [&](const Tile& T, float* sU) {
    const int tid = threadIdx.x;
    float* sF = sU + pad32(BN);
    const SBox<G::HX, G::HY> ub{sU}, fb{sF};
    const SCompact<1> dr{sD};
    auto U = [=](int i, int j) { return sU[T.box<G::HX, G::HY>(i, j)]; };
    auto F = [=](int i, int j) { return sF[T.box<G::HX, G::HY>(i, j)]; };
    // red residual at element e = (rr, pp) of the tile plus 1: fast, or as the per-step
    // kernels (0 off the interior)
    auto red_fast = [=](int e, int rr, int pp) {
      const int a = rr & 1;  // red node of row J0 - 1 + rr
      const int b = ub.template base<1>(rr, pp, a);
      sD[e] = Arith<float>::sub(fb.template get<0, 0>(b, a), cross<EXACT, NT>(c, ub, b, ub, b, a));
    };
    // black node (rr, pp) of the tile = coarse node, residual d: R = 1/2 P^T,
    // Eq. (transfer_r2): terms (0,-1), (-1,0), (0,0), (1,0), (0,1)
    auto coarse = [=](int rr, int pp, float d) {
      const int a = rr & 1;
      const int j = T.J0 + rr, i = 2 * (T.P0 + pp) + a;
      const int bd = dr.template base<0>(rr, pp, a);
      float w = Arith<float>::mul(0.125f, dr.template get<0, -1>(bd, a));
      w = madd<float, EXACT>(w, 0.125f, dr.template get<-1, 0>(bd, a));
      w = madd<float, EXACT>(w, 0.5f, d);
      w = madd<float, EXACT>(w, 0.125f, dr.template get<1, 0>(bd, a));
      const float v = madd<float, EXACT>(w, 0.125f, dr.template get<0, 1>(bd, a));
      const int64_t at = (int64_t)j * pc + (i >> 1);
      fc[at] = v;
      if (TC) tc[at] = (i & 1) ? relax_from_zero(v, node_wd(Lc, i, j)) : 0.f;
    };
    auto black_d = [=](int rr, int pp) {
      const int a = rr & 1;
      const int b = ub.template base<0>(rr, pp, a);
      return Arith<float>::sub(fb.template get<0, 0>(b, a), cross<EXACT, NT>(c, ub, b, ub, b, a));
    };
    auto run = [&](auto check) {
      constexpr bool EDGE = decltype(check)::value;
      // edge tiles walk only the rows that hold fast nodes, then the strips
      const int fa = EDGE ? fast_row0<1>(L, T) : 0;
      const int na = EDGE ? fast_rows<1>(L, T, fa) * Reg<1>::w : Reg<1>::n;
      for (int e = tid; e < na; e += kTT) {
        const int rq = e / Reg<1>::w, pp = e - rq * Reg<1>::w, rr = fa + rq;
        if constexpr (EDGE) {
          int i, j;
          node_of<1>(T, rr, pp, rr & 1, i, j);
          if (!fast_node_c<false>(L, i, j)) continue;
        }
        red_fast(rr * Reg<1>::w + pp, rr, pp);
      }
      if constexpr (EDGE) {  // the nodes outside the fast range, in the strips
        const Strips<1> st(L, T);
        for (int k = tid; k < st.count; k += kTT) {
          int rr, pp;
          st.at(k, rr, pp);
          int i, j;
          node_of<1>(T, rr, pp, rr & 1, i, j);
          if (fast_node_c<false>(L, i, j)) continue;
          sD[rr * Reg<1>::w + pp] =
              inner(n, i, j) ? Arith<float>::sub(F(i, j), stencil<EXACT, NT>(L, c, i, j, U)) : 0.f;
        }
      }
      __syncthreads();
      const int fb0 = EDGE ? fast_row0<0>(L, T) : 0;
      const int nb = EDGE ? fast_rows<0>(L, T, fb0) * kTP : kTJ * kTP;
      for (int e = tid; e < nb; e += kTT) {
        const int rq = e / kTP, pp = e - rq * kTP, rr = fb0 + rq;
        if constexpr (EDGE) {
          int i, j;
          node_of<0>(T, rr, pp, rr & 1, i, j);
          if (!fast_node_c<false>(L, i, j)) continue;
        }
        coarse(rr, pp, black_d(rr, pp));
      }
      if constexpr (EDGE) {
        const Strips<0> st(L, T);
        for (int k = tid; k < st.count; k += kTT) {
          int rr, pp;
          st.at(k, rr, pp);
          int i, j;
          node_of<0>(T, rr, pp, rr & 1, i, j);
          if (fast_node_c<false>(L, i, j) || !inner(n, i, j)) continue;
          coarse(rr, pp, Arith<float>::sub(F(i, j), stencil<EXACT, NT>(L, c, i, j, U)));
        }
      }
    };
    if (fast_tile<1>(L, T)) run(std::false_type{});
    else run(std::true_type{});
  });
}

// ---- rotated levels ----------------------------------------------------------------
// A rotated level's storage row j holds the lattice nodes i = 2q + (j & 1) (q = storage
// column); its red nodes are the odd rows, its black nodes the even rows. A block owns
// kRC storage columns x kRR rows (J0 even). Each colour's values live in compact arrays
// of that colour's rows of a region (M rows and MC columns around the tile, M even).
// The fast stencil is the first Galerkin 9-point one (Eq. L_G1): terms 0-3 (the +-2
// lattice axis neighbours) on rows of the node's colour, terms 4-7 (the diagonal
// neighbours) on the rows of the other colour, term 8 the centre; the host checks this
// shape, and the storage offsets (sdx by row parity, sdy) come from the level.
constexpr int kRC = 128;
constexpr int kRR = 32;

template <int M, int MC>
struct RReg {
  static constexpr int w = kRC + 2 * MC;
  static constexpr int h = kRR / 2 + M;
  static constexpr int n = w * h;
};

struct RTile {
  int J0, C0;
  __device__ RTile(int bx, int by) : J0(by * kRR), C0(bx * kRC) {}
};

// Sources of one colour: RComp (compact rows of parity PAR of a region with margins
// M, MC), RBox (a staged TMA box, both colours, halo HX, HY), RZero (the zero start).
// step2: index distance from a row to the next row of the same colour.
template <int M, int MC, int PAR>
struct RComp {
  float* p;
  static constexpr int step2 = RReg<M, MC>::w;
  __device__ __forceinline__ int idx(const RTile& T, int q, int j) const {
    return ((j - (T.J0 - M) - PAR) >> 1) * RReg<M, MC>::w + (q - (T.C0 - MC));
  }
  // index of the node on row j + DJ (DJ = 0 or -1) above element (kr, cq) of the
  // colour-PN rows of a region (MN, MCN): all offsets compile-time
  template <int MN, int MCN, int PN, int DJ>
  __device__ __forceinline__ int idx_r(int kr, int cq) const {
    static_assert(((PN + DJ + M - MN - PAR) & 1) == 0, "row of this source's colour");
    return (kr + (PN + DJ + M - MN - PAR) / 2) * RReg<M, MC>::w + cq + (MC - MCN);
  }
  __device__ __forceinline__ float at(int k) const { return p[k]; }
};
template <int HX, int HY>
struct RBox {
  const float* p;
  static constexpr int W = kRC + 2 * HX;
  static constexpr int step2 = 2 * W;
  __device__ __forceinline__ int idx(const RTile& T, int q, int j) const {
    return (j - (T.J0 - HY)) * W + (q - (T.C0 - HX));
  }
  template <int MN, int MCN, int PN, int DJ>
  __device__ __forceinline__ int idx_r(int kr, int cq) const {
    return (2 * kr + PN + DJ - MN + HY) * W + cq + (HX - MCN);
  }
  __device__ __forceinline__ float at(int k) const { return p[k]; }
};
struct RZero {
  static constexpr int step2 = 0;
  __device__ __forceinline__ int idx(const RTile&, int, int) const { return 0; }
  template <int MN, int MCN, int PN, int DJ>
  __device__ __forceinline__ int idx_r(int, int) const { return 0; }
  __device__ __forceinline__ float at(int) const { return 0.f; }
};

// The fast stencils of the rotated tile kernels, in evaluation order (lattice offsets):
// 9 points = the first Galerkin stencil (Eq. L_G1): the four (2, 0) neighbours, the four
// diagonal ones, the centre; 25 points = the second rotated Galerkin level of G^(2): the
// four (4, 0), the eight (1, 3), the four (2, 2), the four (2, 0), the four diagonal
// neighbours, the centre. Terms on rows of odd offset are the other colour's.
template <int NT>
__host__ __device__ constexpr int rot_dx(int k) {
  if constexpr (NT == 9) {
    constexpr int x[9] = {0, -2, 2, 0, -1, 1, -1, 1, 0};
    return x[k];
  } else {
    constexpr int x[25] = {0, -4, 4, 0, -1, 1, -3, 3, -3, 3, -1, 1, -2, 2, -2, 2, 0, -2, 2, 0, -1, 1, -1, 1, 0};
    return x[k];
  }
}
template <int NT>
__host__ __device__ constexpr int rot_dy(int k) {
  if constexpr (NT == 9) {
    constexpr int y[9] = {-2, 0, 0, 2, -1, -1, 1, 1, 0};
    return y[k];
  } else {
    constexpr int y[25] = {-4, 0, 0, 4, -3, -3, -1, -1, 1, 1, 3, 3, -2, -2, 2, 2, -2, 0, 0, 2, -1, -1, 1, 1, 0};
    return y[k];
  }
}
template <int NT>
__host__ __device__ constexpr bool rot_gstart(int k) {
  if constexpr (NT == 9) return k == 0 || k == 4 || k == 8;
  else return k == 0 || k == 4 || k == 12 || k == 16 || k == 20 || k == 24;
}
// storage column offset of term k for a node on a row of parity par (i = 2q + par)
template <int NT>
__host__ __device__ constexpr int rot_sdx(int k, int par) {
  return (rot_dy<NT>(k) & 1) ? (2 * par + rot_dx<NT>(k) - 1) / 2 : rot_dx<NT>(k) / 2;
}

// Region margins and box halos of the rotated kernels for a stencil reaching RY rows and
// RX storage columns: each phase's region covers what the next one reads.
template <int NT>
struct RGeo {
  static constexpr int RY = NT == 9 ? 2 : 4, RX = NT == 9 ? 1 : 2;
  static constexpr int M0 = 3 * RY, MC0 = 3 * RX, M1 = 2 * RY, MC1 = 2 * RX, M2 = RY, MC2 = RX;
  static constexpr int PHX = round4(MC0), PHY = M0;        // presmooth: f box
  static constexpr int SHX = round4(2 * RX), SHY = 2 * RY;  // sweep: u, f boxes
  static constexpr int QHX = round4(1 + RX), QHY = 2 + RY;  // residual + restriction
};

// (L x) at a fast node of parity PAR: same-colour terms from ss (base bs = the node),
// other-colour terms from so (base bo = the node's column on row j - 1), in evaluation
// order; every index offset is a compile-time constant.
template <int NT, int PAR, int K, class SS, class SO>
__device__ __forceinline__ float rterm(const SS& ss, int bs, const SO& so, int bo) {
  constexpr int DY = rot_dy<NT>(K), SX = rot_sdx<NT>(K, PAR);
  if constexpr ((DY & 1) != 0) return so.at(bo + ((DY + 1) / 2) * SO::step2 + SX);
  else return ss.at(bs + (DY / 2) * SS::step2 + SX);
}
template <bool EXACT, int NT, int PAR, class SS, class SO, int... K>
__device__ __forceinline__ float rcross_seq(const float (&c)[NT], const SS& ss, int bs, const SO& so, int bo,
                                           std::integer_sequence<int, K...>) {
  const float x[NT] = {rterm<NT, PAR, K>(ss, bs, so, bo)...};
  if constexpr (EXACT) {
    RowSum<float, true> acc;
#pragma unroll
    for (int k = 0; k < NT; ++k) acc.add(c[k], x[k], rot_gstart<NT>(k));
    return acc.value();
  } else {
    float s = Arith<float>::mul(c[0], x[0]);
#pragma unroll
    for (int k = 1; k < NT; ++k) s = Arith<float>::fma(c[k], x[k], s);
    return s;
  }
}
template <bool EXACT, int NT, int PAR, class SS, class SO>
__device__ __forceinline__ float rcross(const float (&c)[NT], const SS& ss, int bs, const SO& so, int bo) {
  return rcross_seq<EXACT, NT, PAR>(c, ss, bs, so, bo, std::make_integer_sequence<int, NT>{});
}

// Value of lattice node (a, b) in a source.
template <class SRC>
__device__ __forceinline__ float rval(const SRC& s, const RTile& T, int a, int b) {
  return s.at(s.idx(T, a >> 1, b));
}

// Strips of the colour-PAR rows of a rotated region (M, MC) that hold its nodes outside
// the fast range (rx <= i <= fxe, ry <= j <= fye), within rows 0 <= j <= n and storage
// columns 0 <= q < cols: compact rows [r0, rt) and [rb, r1), and in the rows between them
// the columns [p0, pl) and [pr, p1). A superset of those nodes, without overlap; nodes
// beyond are never read (fast stencils stay two rows and one column inside, boundary-
// class rows drop boundary columns) nor stored. The fast pass walks rows [rt, rb).
template <int M, int MC, int PAR>
struct RStrips {
  int r0, rt, rb, r1, p0, pl, pr, p1, pw, mw, count;
  __device__ __forceinline__ RStrips(const LevelDev<float>& L, const RTile& T) {
    using G = RReg<M, MC>;
    const int jb = T.J0 - M + PAR, qb = T.C0 - MC;  // row of compact row 0, column of element 0
    // first compact row whose row j = jb + 2 r reaches a bound: (bound - jb) rounded up
    auto first = [&](int bound) { return min(max(bound - jb + 1, 0) >> 1, G::h); };
    r0 = first(0);
    r1 = max(r0, first(L.n + 1));
    rt = min(max(first(L.ry), r0), r1);
    rb = min(max(first(L.fye + 1), rt), r1);
    p0 = min(max(-qb, 0), G::w);
    p1 = max(p0, min(L.cols - qb, G::w));
    pl = min(max(L.rx / 2 + 1 - qb, p0), p1);           // i = 2q + PAR < rx only if q <= rx / 2
    pr = max(pl, min(max((L.fxe - 1) / 2 - qb, p0), p1));  // ... i > fxe only if q >= (fxe - 1) / 2
    pw = p1 - p0;
    mw = (pl - p0) + (p1 - pr);
    count = (rt - r0 + r1 - rb) * pw + (rb - rt) * mw;
  }
  __device__ __forceinline__ void at(int k, int& kr, int& cq) const {
    const int k1 = (rt - r0) * pw, k2 = k1 + (r1 - rb) * pw;
    if (k < k1) {
      const int q = k / pw;
      kr = r0 + q;
      cq = p0 + (k - q * pw);
    } else if (k < k2) {
      const int q = (k - k1) / pw;
      kr = rb + q;
      cq = p0 + (k - k1 - q * pw);
    } else {
      const int q = (k - k2) / mw, r = k - k2 - q * mw;
      kr = rt + q;
      cq = r < pl - p0 ? p0 + r : pr + (r - (pl - p0));
    }
  }
};

// One relaxation phase over the nodes of colour PAR in the region (M, MC): the fast
// value (relax of the fast stencil, or 0 + f omega / a_pp with ZERO) for nodes of the
// fast range; with EDGE (a tile reaching the boundary strip) only the rows holding fast
// nodes are walked with the fast stencil, and the strip nodes outside the fast range
// get gen(i, j) in a second pass. sink(e, q, j, v), e = index in the region's array.
template <bool EXACT, int NT, int PAR, int M, int MC, bool ZERO, bool EDGE, class SS, class SO, class FB, class SINK,
          class GEN>
__device__ __forceinline__ void rphase(const float (&c)[NT], float wd, const SS& ss, const SO& so, const FB& fb,
                                       const RTile& T, const LevelDev<float>& L, SINK sink, GEN gen) {
  using G = RReg<M, MC>;
  auto fast = [&](int e, int kr, int cq) {
    const int j = T.J0 - M + 2 * kr + PAR, q = T.C0 - MC + cq;
    if (EDGE && !fast_node_c<false>(L, 2 * q + PAR, j)) return;
    const float f = fb.at(fb.template idx_r<M, MC, PAR, 0>(kr, cq));
    float v;
    if constexpr (ZERO) {
      v = relax_from_zero(f, wd);
    } else {
      const int bs = ss.template idx_r<M, MC, PAR, 0>(kr, cq);
      v = relax<EXACT>(rcross<EXACT, NT, PAR>(c, ss, bs, so, so.template idx_r<M, MC, PAR, -1>(kr, cq)), f, ss.at(bs),
                       wd);
    }
    sink(e, q, j, v);
  };
  if constexpr (!EDGE) {
    for (int e = threadIdx.x; e < G::n; e += kTT) {
      const int kr = e / G::w;
      fast(e, kr, e - kr * G::w);
    }
  } else {
    const RStrips<M, MC, PAR> st(L, T);
    for (int e = threadIdx.x; e < (st.rb - st.rt) * G::w; e += kTT) {
      const int r = e / G::w, kr = st.rt + r, cq = e - r * G::w;
      fast(kr * G::w + cq, kr, cq);
    }
    for (int k = threadIdx.x; k < st.count; k += kTT) {
      int kr, cq;
      st.at(k, kr, cq);
      const int j = T.J0 - M + 2 * kr + PAR, q = T.C0 - MC + cq;
      if (fast_node_c<false>(L, 2 * q + PAR, j)) continue;
      sink(kr * G::w + cq, q, j, gen(2 * q + PAR, j));
    }
  }
}

// Whether every node of the region (M, MC) is in the fast range of the rotated level L.
template <int M, int MC>
__device__ __forceinline__ bool rfast_tile(const LevelDev<float>& L, const RTile& T) {
  return 2 * (T.C0 - MC) >= L.rx && 2 * (T.C0 + kRC + MC - 1) + 1 <= L.fxe && T.J0 - M >= L.ry &&
         T.J0 + kRR - 1 + M <= L.fye;
}

template <int NB, class BODY>
__device__ __forceinline__ void rtile_block(float* box0, int box_floats, const CUtensorMap* const (&maps)[NB], int hx,
                                            int hy, int* status, BODY body) {
  __shared__ uint64_t bar;
  const RTile T(blockIdx.x, blockIdx.y);
  if (threadIdx.x == 0) {
    mbar_init(&bar);
    mbar_expect(&bar, (uint32_t)(NB * (kRC + 2 * hx) * (kRR + 2 * hy) * sizeof(float)));
#pragma unroll
    for (int m = 0; m < NB; ++m) tma_load(box0 + m * box_floats, maps[m], T.C0 - hx, T.J0 - hy, &bar);
  }
  __syncthreads();
  if (!wait_tile(&bar, status)) return;
  body(T, box0);
}

// Store row j of the tile (values from the compact array src of that row's colour) to
// the level's storage, bounds-checked.
template <class SRC>
__device__ __forceinline__ void rstore_row(float* out, const LevelDev<float>& L, const RTile& T, const SRC& src, int j,
                                           int cq) {
  const int q = T.C0 + cq;
  if (j > L.n || q >= L.cols) return;
  out[(int64_t)j * L.pitch + q] = src.at(src.idx(T, q, j));
}

// ---- rotated presmooth: 2 red-black sweeps from u = 0 ------------------------------
template <bool EXACT, int NT>
__global__ void __launch_bounds__(kTT, 3) k_rtile_presmooth(const LevelDev<float>* __restrict__ Lp,
                                                         const __grid_constant__ CUtensorMap mapF,
                                                         float* __restrict__ out, int* __restrict__ status) {
  using G = RGeo<NT>;
  constexpr int FN = (kRC + 2 * G::PHX) * (kRR + 2 * G::PHY);
  extern __shared__ __align__(128) unsigned char tile_smem[];
  float* box0 = smem_base(tile_smem);
  float* sR0 = box0 + pad32(FN);
  float* sB1 = sR0 + RReg<G::M0, G::MC0>::n;
  float* sR2 = sB1 + RReg<G::M1, G::MC1>::n;
  const LevelDev<float>& L = *Lp;
  float c[NT];
#pragma unroll
  for (int k = 0; k < NT; ++k) c[k] = L.c[k];
  const float wdf = L.wd;
  const int n = L.n;
  const CUtensorMap* const maps[1] = {&mapF};
  rtile_block<1>(box0, pad32(FN), maps, G::PHX, G::PHY, status, [&](const RTile& T, float* sF) {
    const RBox<G::PHX, G::PHY> fb{sF};
    const RComp<G::M0, G::MC0, 1> r0{sR0};
    const RComp<G::M1, G::MC1, 0> b1{sB1};
    const RComp<G::M2, G::MC2, 1> r2{sR2};
    auto F = [=](int i, int j) { return rval(fb, T, i, j); };
    auto run = [&](auto check) {
      constexpr bool EDGE = decltype(check)::value;
      // red from zero: 0 + f omega / a_pp
      rphase<EXACT, NT, 1, G::M0, G::MC0, true, EDGE>(c, wdf, RZero{}, RZero{}, fb, T, L,
                                         [=](int e, int, int, float v) { sR0[e] = v; }, [=](int i, int j) {
                                           return inner(n, i, j) ? relax_from_zero(F(i, j), wd_at(L, wdf, i, j)) : 0.f;
                                         });
      __syncthreads();
      // black of sweep 1 (old values 0)
      rphase<EXACT, NT, 0, G::M1, G::MC1, false, EDGE>(c, wdf, RZero{}, r0, fb, T, L, [=](int e, int, int, float v) { sB1[e] = v; },
                                          [=](int i, int j) {
                                            if (!inner(n, i, j)) return 0.f;
                                            const float st = class_stencil<EXACT>(L, i, j, [=](int a, int b) {
                                              return (a & 1) ? rval(r0, T, a, b) : 0.f;
                                            });
                                            return relax<EXACT>(st, F(i, j), 0.f, wd_at(L, wdf, i, j));
                                          });
      __syncthreads();
      // red of sweep 2
      rphase<EXACT, NT, 1, G::M2, G::MC2, false, EDGE>(c, wdf, r0, b1, fb, T, L, [=](int e, int, int, float v) { sR2[e] = v; },
                                          [=](int i, int j) {
                                            if (!inner(n, i, j)) return 0.f;
                                            const float st = class_stencil<EXACT>(L, i, j, [=](int a, int b) {
                                              return (a & 1) ? rval(r0, T, a, b) : rval(b1, T, a, b);
                                            });
                                            return relax<EXACT>(st, F(i, j), rval(r0, T, i, j), wd_at(L, wdf, i, j));
                                          });
      __syncthreads();
      // black of sweep 2 on the tile, stored; then the red rows of the tile
      rphase<EXACT, NT, 0, 0, 0, false, EDGE>(
          c, wdf, b1, r2, fb, T, L,
          [=](int, int q, int j, float v) {
            if (EDGE && (j > n || q >= L.cols)) return;
            out[(int64_t)j * L.pitch + q] = v;
          },
          [=](int i, int j) {
            if (!inner(n, i, j)) return 0.f;
            const float st = class_stencil<EXACT>(L, i, j, [=](int a, int b) {
              return (a & 1) ? rval(r2, T, a, b) : rval(b1, T, a, b);
            });
            return relax<EXACT>(st, F(i, j), rval(b1, T, i, j), wd_at(L, wdf, i, j));
          });
      for (int e = threadIdx.x; e < (kRR / 2) * kRC; e += kTT) {
        const int kr = e / kRC, cq = e - kr * kRC;
        rstore_row(out, L, T, r2, T.J0 + 2 * kr + 1, cq);
      }
    };
    if (rfast_tile<G::M0, G::MC0>(L, T)) run(std::false_type{});
    else run(std::true_type{});
  });
}

// ---- rotated sweep: one red-black sweep, u -> out ------------------------------------
template <bool EXACT, int NT>
__global__ void __launch_bounds__(kTT, 3) k_rtile_sweep(const LevelDev<float>* __restrict__ Lp,
                                                     const __grid_constant__ CUtensorMap mapU,
                                                     const __grid_constant__ CUtensorMap mapF, float* __restrict__ out,
                                                     int* __restrict__ status) {
  using G = RGeo<NT>;
  constexpr int BN = (kRC + 2 * G::SHX) * (kRR + 2 * G::SHY);
  extern __shared__ __align__(128) unsigned char tile_smem[];
  float* box0 = smem_base(tile_smem);
  float* sR = box0 + 2 * pad32(BN);
  const LevelDev<float>& L = *Lp;
  float c[NT];
#pragma unroll
  for (int k = 0; k < NT; ++k) c[k] = L.c[k];
  const float wdf = L.wd;
  const int n = L.n;
  const CUtensorMap* const maps[2] = {&mapU, &mapF};
  rtile_block<2>(box0, pad32(BN), maps, G::SHX, G::SHY, status, [&](const RTile& T, float* sU) {
    const RBox<G::SHX, G::SHY> ub{sU}, fb{sU + pad32(BN)};
    const RComp<G::M2, G::MC2, 1> rn{sR};
    auto U = [=](int i, int j) { return rval(ub, T, i, j); };
    auto F = [=](int i, int j) { return rval(fb, T, i, j); };
    auto run = [&](auto check) {
      constexpr bool EDGE = decltype(check)::value;
      rphase<EXACT, NT, 1, G::M2, G::MC2, false, EDGE>(c, wdf, ub, ub, fb, T, L, [=](int e, int, int, float v) { sR[e] = v; },
                                          [=](int i, int j) {
                                            const float v = U(i, j);
                                            return inner(n, i, j) ? relax<EXACT>(class_stencil<EXACT>(L, i, j, U),
                                                                                 F(i, j), v, wd_at(L, wdf, i, j))
                                                                  : v;
                                          });
      __syncthreads();
      rphase<EXACT, NT, 0, 0, 0, false, EDGE>(
          c, wdf, ub, rn, fb, T, L,
          [=](int, int q, int j, float v) {
            if (EDGE && (j > n || q >= L.cols)) return;
            out[(int64_t)j * L.pitch + q] = v;
          },
          [=](int i, int j) {
            const float v = U(i, j);
            if (!inner(n, i, j)) return v;
            const float st = class_stencil<EXACT>(L, i, j, [=](int a, int b) {
              return (a & 1) ? rval(rn, T, a, b) : U(a, b);
            });
            return relax<EXACT>(st, F(i, j), v, wd_at(L, wdf, i, j));
          });
      for (int e = threadIdx.x; e < (kRR / 2) * kRC; e += kTT) {
        const int kr = e / kRC, cq = e - kr * kRC;
        rstore_row(out, L, T, rn, T.J0 + 2 * kr + 1, cq);
      }
    };
    if (rfast_tile<G::M2, G::MC2>(L, T)) run(std::false_type{});
    else run(std::true_type{});
  });
}

// ---- rotated residual + red-black restriction (rotated level -> its axis level) ------
// Coarse nodes = the black (even-row) nodes; R = 1/2 P^T, Eq. (transfer_r2) in the
// rotated frame: terms (-1,-1), (1,-1), (0,0), (-1,1), (1,1) (lattice offsets).
template <bool EXACT, int NT, bool TC>
__global__ void __launch_bounds__(kTT, 3) k_rtile_res_restrict(const LevelDev<float>* __restrict__ Lp,
                                                            const LevelDev<float>* __restrict__ Lcp,
                                                            const __grid_constant__ CUtensorMap mapU,
                                                            const __grid_constant__ CUtensorMap mapF,
                                                            float* __restrict__ fc, float* __restrict__ tc,
                                                            int* __restrict__ status) {
  using G = RGeo<NT>;
  constexpr int BN = (kRC + 2 * G::QHX) * (kRR + 2 * G::QHY);
  extern __shared__ __align__(128) unsigned char tile_smem[];
  float* box0 = smem_base(tile_smem);
  float* sD = box0 + 2 * pad32(BN);  // residuals of the red nodes, region (2, 1)
  const LevelDev<float>& L = *Lp;
  const LevelDev<float>& Lc = *Lcp;
  float c[NT];
#pragma unroll
  for (int k = 0; k < NT; ++k) c[k] = L.c[k];
  const int n = L.n, pc = Lc.pitch;
  const CUtensorMap* const maps[2] = {&mapU, &mapF};
  rtile_block<2>(box0, pad32(BN), maps, G::QHX, G::QHY, status, [&](const RTile& T, float* sU) {
    const RBox<G::QHX, G::QHY> ub{sU}, fb{sU + pad32(BN)};
    const RComp<2, 1, 1> dr{sD};
    auto U = [=](int i, int j) { return rval(ub, T, i, j); };
    auto F = [=](int i, int j) { return rval(fb, T, i, j); };
    auto run = [&](auto check) {
      constexpr bool EDGE = decltype(check)::value;
      // red residuals on the region (2, 1) (0 off the interior), through the phase walker
      // with a residual in place of the relaxation
      using G = RReg<2, 1>;
      auto red_fast = [&](int e, int kr, int cq) {
        const int j = T.J0 - 2 + 2 * kr + 1, q = T.C0 - 1 + cq;
        if (EDGE && !fast_node_c<false>(L, 2 * q + 1, j)) return;
        const int b = ub.idx(T, q, j);
        sD[e] = Arith<float>::sub(fb.at(fb.idx(T, q, j)), rcross<EXACT, NT, 1>(c, ub, b, ub, ub.idx(T, q, j - 1)));
      };
      if constexpr (!EDGE) {
        for (int e = threadIdx.x; e < G::n; e += kTT) {
          const int kr = e / G::w;
          red_fast(e, kr, e - kr * G::w);
        }
      } else {
        const RStrips<2, 1, 1> st(L, T);
        for (int e = threadIdx.x; e < (st.rb - st.rt) * G::w; e += kTT) {
          const int r = e / G::w, kr = st.rt + r, cq = e - r * G::w;
          red_fast(kr * G::w + cq, kr, cq);
        }
        for (int k = threadIdx.x; k < st.count; k += kTT) {
          int kr, cq;
          st.at(k, kr, cq);
          const int j = T.J0 - 2 + 2 * kr + 1, q = T.C0 - 1 + cq, i = 2 * q + 1;
          if (fast_node_c<false>(L, i, j)) continue;
          sD[kr * G::w + cq] = inner(n, i, j) ? Arith<float>::sub(F(i, j), class_stencil<EXACT>(L, i, j, U)) : 0.f;
        }
      }
      __syncthreads();
      // black nodes of the tile = coarse nodes
      auto coarse = [&](int q, int j, float d) {
        const int bu = dr.idx(T, q, j - 1);  // red row j - 1, columns q - 1 and q; then row j + 1
        float w = Arith<float>::mul(0.125f, dr.at(bu - 1));
        w = madd<float, EXACT>(w, 0.125f, dr.at(bu));
        w = madd<float, EXACT>(w, 0.5f, d);
        w = madd<float, EXACT>(w, 0.125f, dr.at(bu + G::w - 1));
        const float v = madd<float, EXACT>(w, 0.125f, dr.at(bu + G::w));
        const int I = q, J = j >> 1;  // the coarse (axis) node
        const int64_t at = (int64_t)J * pc + I;
        fc[at] = v;
        if (TC) tc[at] = ((I + J) & 1) ? relax_from_zero(v, node_wd(Lc, I, J)) : 0.f;
      };
      auto black_fast = [&](int kr, int cq) {
        const int j = T.J0 + 2 * kr, q = T.C0 + cq;
        if (EDGE && !fast_node_c<false>(L, 2 * q, j)) return;
        coarse(q, j,
               Arith<float>::sub(fb.at(fb.idx(T, q, j)), rcross<EXACT, NT, 0>(c, ub, ub.idx(T, q, j), ub, ub.idx(T, q, j - 1))));
      };
      using G0 = RReg<0, 0>;
      if constexpr (!EDGE) {
        for (int e = threadIdx.x; e < G0::n; e += kTT) {
          const int kr = e / G0::w;
          black_fast(kr, e - kr * G0::w);
        }
      } else {
        const RStrips<0, 0, 0> st(L, T);
        for (int e = threadIdx.x; e < (st.rb - st.rt) * G0::w; e += kTT) {
          const int r = e / G0::w;
          black_fast(st.rt + r, e - r * G0::w);
        }
        for (int k = threadIdx.x; k < st.count; k += kTT) {
          int kr, cq;
          st.at(k, kr, cq);
          const int j = T.J0 + 2 * kr, q = T.C0 + cq, i = 2 * q;
          if (fast_node_c<false>(L, i, j) || !inner(n, i, j)) continue;
          coarse(q, j, Arith<float>::sub(F(i, j), class_stencil<EXACT>(L, i, j, U)));
        }
      }
    };
    if (rfast_tile<2, 1>(L, T)) run(std::false_type{});
    else run(std::true_type{});
  });
}

// ---- host side -----------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// 2D map over a level's (n + 1) x (n + 1) nodes (row stride pitch) with a box of
// (kTQ + 2 hx) x (kTJ + 2 hy) elements.
bool make_map(CUtensorMap* m, const float* base, const LevelDev<float>& L, int hx, int hy, int tw = kTQ,
              int th = kTJ) {
  const auto enc = tensor_map_encoder();
  if (!enc) return false;
  std::memset(m, 0, sizeof(*m));
  const cuuint64_t dims[2] = {(cuuint64_t)L.cols, (cuuint64_t)L.rows};
  const cuuint64_t strides[1] = {(cuuint64_t)L.pitch * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)(tw + 2 * hx), (cuuint32_t)(th + 2 * hy)};
  const cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Dynamic shared memory of each kernel: its staged boxes (each padded to 32 floats), its
// one-colour arrays, and 128 bytes to align the base.
template <int R, int NS>
size_t pre_smem() {
  using G = PreGeo<R, NS>;
  size_t n = (size_t)pad32((kTQ + 2 * G::HX) * (kTJ + 2 * G::HY)) + Reg<G::M0>::n;
  if (NS == 2) n += Reg<2 * R>::n + Reg<R>::n;
  return n * sizeof(float) + 128;
}
template <int R>
size_t sweep_smem() {
  using G = SweepGeo<R>;
  return (2 * (size_t)pad32((kTQ + 2 * G::HX) * (kTJ + 2 * G::HY)) + Reg<R>::n) * sizeof(float) + 128;
}
template <int R>
size_t rr_smem() {
  using G = RrGeo<R>;
  return (2 * (size_t)pad32((kTQ + 2 * G::HX) * (kTJ + 2 * G::HY)) + Reg<1>::n) * sizeof(float) + 128;
}

template <int NT>
size_t rpre_smem() {
  using G = RGeo<NT>;
  return ((size_t)pad32((kRC + 2 * G::PHX) * (kRR + 2 * G::PHY)) + RReg<G::M0, G::MC0>::n + RReg<G::M1, G::MC1>::n +
          RReg<G::M2, G::MC2>::n) *
             sizeof(float) +
         128;
}
template <int NT>
size_t rsw_smem() {
  using G = RGeo<NT>;
  return (2 * (size_t)pad32((kRC + 2 * G::SHX) * (kRR + 2 * G::SHY)) + RReg<G::M2, G::MC2>::n) * sizeof(float) + 128;
}
template <int NT>
size_t rrr_smem() {
  using G = RGeo<NT>;
  return (2 * (size_t)pad32((kRC + 2 * G::QHX) * (kRR + 2 * G::QHY)) + RReg<2, 1>::n) * sizeof(float) + 128;
}

// Raise a kernel's dynamic shared-memory limit once per process (the sizes are fixed
// per instantiation).
template <auto KERNEL>
cudaError_t allow_smem(size_t bytes) {
  static const cudaError_t e = cudaFuncSetAttribute(KERNEL, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return e;
}

}  // namespace

// Rotated levels: one of the stencils of rot_dx / rot_dy in evaluation order (the first
// Galerkin 9-point stencil, or the 25-point one of the second rotated Galerkin level).
template <int NT>
bool rot_shape_is(const LevelDev<float>& L) {
  if (L.nt != NT) return false;
  for (int k = 0; k < kMaxTerms; ++k) {
    const bool start = (L.gmask[k >> 5] >> (k & 31)) & 1u;
    if (k >= NT ? start : start != rot_gstart<NT>(k)) return false;
  }
  for (int k = 0; k < NT; ++k)
    if (L.sdy[k] != rot_dy<NT>(k) || L.sdx[0][k] != rot_sdx<NT>(k, 0) || L.sdx[1][k] != rot_sdx<NT>(k, 1)) return false;
  return true;
}
bool rot_tile_shape(const LevelDev<float>& L) { return rot_shape_is<9>(L) || rot_shape_is<25>(L); }

bool gbit_host(const uint32_t* m, int k) { return (m[k >> 5] >> (k & 31)) & 1u; }

bool tile_eligible(const LevelPair<float>& P) {
  const LevelDev<float>& L = P.h;
  if (L.per || L.bf16 || L.rows < kTileMinRows) return false;
  if (L.pitch % 4 != 0) return false;  // TMA row stride: 16 bytes
  if (L.kind == kRot) return rot_tile_shape(L);
  if (L.kind != kAxis) return false;
  // the fast stencil must be the 5-point or 9-point cross with terms in (dy, dx) order
  // (offsets in evaluation order: groups of equal coefficient, see LevelDev::c)
  static const int x5[5] = {0, -1, 1, 0, 0}, y5[5] = {-1, 0, 0, 1, 0};
  static const int x9[9] = {0, -2, 2, 0, 0, -1, 1, 0, 0}, y9[9] = {-2, 0, 0, 2, -1, 0, 0, 1, 0};
  if (wide_nt(L.nt)) {  // the second and third red-black Galerkin axis levels
    for (int k = 0; k < L.nt; ++k) {
      const bool ok = L.nt == 21 ? L.sdx[0][k] == wide_dx<21>(k) && L.sdy[k] == wide_dy<21>(k) &&
                                       gbit_host(L.gmask, k) == wide_gstart<21>(k)
                                 : L.sdx[0][k] == wide_dx<37>(k) && L.sdy[k] == wide_dy<37>(k) &&
                                       gbit_host(L.gmask, k) == wide_gstart<37>(k);
      if (!ok) return false;
    }
    for (int k = L.nt; k < kMaxTerms; ++k)
      if (gbit_host(L.gmask, k)) return false;
    return true;
  } else {
    const int* xs = L.nt == 5 ? x5 : L.nt == 9 ? x9 : nullptr;
    const int* ys = L.nt == 5 ? y5 : y9;
    if (!xs) return false;
    for (int k = 0; k < L.nt; ++k)
      if (L.sdx[0][k] != xs[k] || L.sdy[k] != ys[k]) return false;
    if (L.gmask[0] != fast_gmask(L.nt)) return false;
  }
  for (int w = 1; w < kMaxTerms / 32; ++w)
    if (L.gmask[w]) return false;
  return true;
}

namespace {
// Tensor maps of a rotated level with the NT-point stencil.
template <int NT>
bool rot_maps(TileLevel& T, const LevelDev<float>& L, float* u, float* t, float* f) {
  using G = RGeo<NT>;
  bool ok = true;
  if (T.nu1) ok &= make_map(&T.f_pre, f, L, G::PHX, G::PHY, kRC, kRR);
  ok &= make_map(&T.u_sw, u, L, G::SHX, G::SHY, kRC, kRR);
  ok &= make_map(&T.t_sw, t, L, G::SHX, G::SHY, kRC, kRR);
  ok &= make_map(&T.f_sw, f, L, G::SHX, G::SHY, kRC, kRR);
  ok &= make_map(&T.u_rr, u, L, G::QHX, G::QHY, kRC, kRR);
  ok &= make_map(&T.f_rr, f, L, G::QHX, G::QHY, kRC, kRR);
  return ok;
}

// Tensor maps of an axis level whose fast stencil reaches R nodes.
template <int R>
bool axis_maps(TileLevel& T, const LevelDev<float>& L, float* u, float* t, float* f) {
  bool ok = true;
  if (T.nu1 == 2) ok &= make_map(&T.f_pre, f, L, PreGeo<R, 2>::HX, PreGeo<R, 2>::HY);
  if (T.nu1 == 1) ok &= make_map(&T.f_pre, f, L, PreGeo<R, 1>::HX, PreGeo<R, 1>::HY);
  ok &= make_map(&T.u_sw, u, L, SweepGeo<R>::HX, SweepGeo<R>::HY);
  ok &= make_map(&T.t_sw, t, L, SweepGeo<R>::HX, SweepGeo<R>::HY);
  ok &= make_map(&T.f_sw, f, L, SweepGeo<R>::HX, SweepGeo<R>::HY);
  ok &= make_map(&T.u_rr, u, L, RrGeo<R>::HX, RrGeo<R>::HY);
  ok &= make_map(&T.f_rr, f, L, RrGeo<R>::HX, RrGeo<R>::HY);
  return ok;
}
}  // namespace

// Multiprocessors of the current device.
int device_sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return n;
}

bool tile_setup(TileLevel& T, const LevelPair<float>& P, float* u, float* t, float* f, int nu1) {
  T.on = false;
  if (!tile_eligible(P)) return false;
  const LevelDev<float>& L = P.h;
  // The wide stencils' tiles carry several times the work of a cross stencil's: below one
  // tile per multiprocessor the per-step kernels, which spread a level over every SM,
  // were faster (measured on GB300: 1025^2 mixed solve 4.04 ms with per-step kernels on
  // its 21- and 37-point levels, 4.20 ms with 85 and 27 tiles there).
  if (wide_nt(L.nt) && (long)((L.cols + kTQ - 1) / kTQ) * ((L.rows + kTJ - 1) / kTJ) < device_sms()) return false;
  T.nt = L.nt;
  T.reach = tile_reach(L.nt);
  T.rot = L.kind == kRot;
  bool ok = true;
  if (T.rot) {  // rotated tiles: presmooth for nu1 = 2 only
    T.nu1 = nu1 == 2 ? 2 : 0;
    T.grid = dim3((L.cols + kRC - 1) / kRC, (L.rows + kRR - 1) / kRR);
    if (L.nt == 25 && (long)T.grid.x * T.grid.y < device_sms()) return false;  // as for the axis wide stencils
    ok &= L.nt == 9 ? rot_maps<9>(T, L, u, t, f) : rot_maps<25>(T, L, u, t, f);
    T.on = ok;
    return ok;
  }
  T.nu1 = (nu1 == 1 || nu1 == 2) ? nu1 : 0;
  T.grid = dim3((L.cols + kTQ - 1) / kTQ, (L.rows + kTJ - 1) / kTJ);
  if (T.reach == 3) ok &= axis_maps<3>(T, L, u, t, f);
  else if (T.reach == 2) ok &= axis_maps<2>(T, L, u, t, f);
  else ok &= axis_maps<1>(T, L, u, t, f);
  T.on = ok;
  return ok;
}

namespace {
template <bool EXACT, int NT, int NS>
cudaError_t presmooth_as(const TileLevel& T, const LevelPair<float>& L, float* u, int* status, cudaStream_t s) {
  const size_t smem = pre_smem<tile_reach(NT), NS>();
  cudaError_t e = allow_smem<k_tile_presmooth<EXACT, NT, NS>>(smem);
  if (e != cudaSuccess) return e;
  k_tile_presmooth<EXACT, NT, NS><<<T.grid, kTT, smem, s>>>(L.d, T.f_pre, u, status);
  return cudaGetLastError();
}
template <bool EXACT, int NT>
cudaError_t sweep_as(const TileLevel& T, const LevelPair<float>& L, bool from_t, float* out, int* status,
                     cudaStream_t s) {
  const size_t smem = sweep_smem<tile_reach(NT)>();
  cudaError_t e = allow_smem<k_tile_sweep<EXACT, NT>>(smem);
  if (e != cudaSuccess) return e;
  k_tile_sweep<EXACT, NT><<<T.grid, kTT, smem, s>>>(L.d, from_t ? T.t_sw : T.u_sw, T.f_sw, out, status);
  return cudaGetLastError();
}
template <bool EXACT, int NT, bool TC>
cudaError_t rr_as(const TileLevel& T, const LevelPair<float>& L, const LevelPair<float>& Lc, float* fc, float* tc,
                  int* status, cudaStream_t s) {
  const size_t smem = rr_smem<tile_reach(NT)>();
  cudaError_t e = allow_smem<k_tile_res_restrict<EXACT, NT, TC>>(smem);
  if (e != cudaSuccess) return e;
  k_tile_res_restrict<EXACT, NT, TC><<<T.grid, kTT, smem, s>>>(L.d, Lc.d, T.u_rr, T.f_rr, fc, tc, status);
  return cudaGetLastError();
}
}  // namespace

namespace {
template <bool EXACT, int NT>
cudaError_t rpresmooth_as(const TileLevel& T, const LevelPair<float>& L, float* u, int* status, cudaStream_t s) {
  const size_t smem = rpre_smem<NT>();
  cudaError_t e = allow_smem<k_rtile_presmooth<EXACT, NT>>(smem);
  if (e != cudaSuccess) return e;
  k_rtile_presmooth<EXACT, NT><<<T.grid, kTT, smem, s>>>(L.d, T.f_pre, u, status);
  return cudaGetLastError();
}
template <bool EXACT, int NT>
cudaError_t rsweep_as(const TileLevel& T, const LevelPair<float>& L, bool from_t, float* out, int* status,
                      cudaStream_t s) {
  const size_t smem = rsw_smem<NT>();
  cudaError_t e = allow_smem<k_rtile_sweep<EXACT, NT>>(smem);
  if (e != cudaSuccess) return e;
  k_rtile_sweep<EXACT, NT><<<T.grid, kTT, smem, s>>>(L.d, from_t ? T.t_sw : T.u_sw, T.f_sw, out, status);
  return cudaGetLastError();
}
template <bool EXACT, int NT, bool TC>
cudaError_t rrr_as(const TileLevel& T, const LevelPair<float>& L, const LevelPair<float>& Lc, float* fc, float* tc,
                   int* status, cudaStream_t s) {
  const size_t smem = rrr_smem<NT>();
  cudaError_t e = allow_smem<k_rtile_res_restrict<EXACT, NT, TC>>(smem);
  if (e != cudaSuccess) return e;
  k_rtile_res_restrict<EXACT, NT, TC><<<T.grid, kTT, smem, s>>>(L.d, Lc.d, T.u_rr, T.f_rr, fc, tc, status);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_tile_presmooth(const TileLevel& T, const LevelPair<float>& L, bool exact, float* u, int* status,
                                  cudaStream_t s) {
  if (!T.on || !T.nu1) return cudaErrorInvalidValue;
  if (T.rot) {
    if (T.nt == 25) return exact ? rpresmooth_as<true, 25>(T, L, u, status, s) : rpresmooth_as<false, 25>(T, L, u, status, s);
    return exact ? rpresmooth_as<true, 9>(T, L, u, status, s) : rpresmooth_as<false, 9>(T, L, u, status, s);
  }
  if (T.nt == 21) {
    if (T.nu1 == 2) return exact ? presmooth_as<true, 21, 2>(T, L, u, status, s) : presmooth_as<false, 21, 2>(T, L, u, status, s);
    return exact ? presmooth_as<true, 21, 1>(T, L, u, status, s) : presmooth_as<false, 21, 1>(T, L, u, status, s);
  }
  if (T.nt == 37) {
    if (T.nu1 == 2) return exact ? presmooth_as<true, 37, 2>(T, L, u, status, s) : presmooth_as<false, 37, 2>(T, L, u, status, s);
    return exact ? presmooth_as<true, 37, 1>(T, L, u, status, s) : presmooth_as<false, 37, 1>(T, L, u, status, s);
  }
  if (T.nt == 9) {
    if (T.nu1 == 2) return exact ? presmooth_as<true, 9, 2>(T, L, u, status, s) : presmooth_as<false, 9, 2>(T, L, u, status, s);
    return exact ? presmooth_as<true, 9, 1>(T, L, u, status, s) : presmooth_as<false, 9, 1>(T, L, u, status, s);
  }
  if (T.nu1 == 2) return exact ? presmooth_as<true, 5, 2>(T, L, u, status, s) : presmooth_as<false, 5, 2>(T, L, u, status, s);
  return exact ? presmooth_as<true, 5, 1>(T, L, u, status, s) : presmooth_as<false, 5, 1>(T, L, u, status, s);
}

cudaError_t launch_tile_sweep(const TileLevel& T, const LevelPair<float>& L, bool exact, bool from_t, float* uout,
                              int* status, cudaStream_t s) {
  if (!T.on) return cudaErrorInvalidValue;
  if (T.rot) {
    if (T.nt == 25)
      return exact ? rsweep_as<true, 25>(T, L, from_t, uout, status, s) : rsweep_as<false, 25>(T, L, from_t, uout, status, s);
    return exact ? rsweep_as<true, 9>(T, L, from_t, uout, status, s) : rsweep_as<false, 9>(T, L, from_t, uout, status, s);
  }
  if (T.nt == 21)
    return exact ? sweep_as<true, 21>(T, L, from_t, uout, status, s) : sweep_as<false, 21>(T, L, from_t, uout, status, s);
  if (T.nt == 37)
    return exact ? sweep_as<true, 37>(T, L, from_t, uout, status, s) : sweep_as<false, 37>(T, L, from_t, uout, status, s);
  if (T.nt == 9)
    return exact ? sweep_as<true, 9>(T, L, from_t, uout, status, s) : sweep_as<false, 9>(T, L, from_t, uout, status, s);
  return exact ? sweep_as<true, 5>(T, L, from_t, uout, status, s) : sweep_as<false, 5>(T, L, from_t, uout, status, s);
}

cudaError_t launch_tile_res_restrict(const TileLevel& T, const LevelPair<float>& L, const LevelPair<float>& Lc,
                                     bool exact, float* fc, float* tc, int* status, cudaStream_t s) {
  if (!T.on || Lc.h.bf16) return cudaErrorInvalidValue;
  if (T.rot) {
    if (Lc.h.kind != kAxis) return cudaErrorInvalidValue;
    if (T.nt == 25) {
      if (tc) return exact ? rrr_as<true, 25, true>(T, L, Lc, fc, tc, status, s) : rrr_as<false, 25, true>(T, L, Lc, fc, tc, status, s);
      return exact ? rrr_as<true, 25, false>(T, L, Lc, fc, tc, status, s) : rrr_as<false, 25, false>(T, L, Lc, fc, tc, status, s);
    }
    if (tc) return exact ? rrr_as<true, 9, true>(T, L, Lc, fc, tc, status, s) : rrr_as<false, 9, true>(T, L, Lc, fc, tc, status, s);
    return exact ? rrr_as<true, 9, false>(T, L, Lc, fc, tc, status, s) : rrr_as<false, 9, false>(T, L, Lc, fc, tc, status, s);
  }
  if (Lc.h.kind != kRot) return cudaErrorInvalidValue;
  if (T.nt == 21) {
    if (tc) return exact ? rr_as<true, 21, true>(T, L, Lc, fc, tc, status, s) : rr_as<false, 21, true>(T, L, Lc, fc, tc, status, s);
    return exact ? rr_as<true, 21, false>(T, L, Lc, fc, tc, status, s) : rr_as<false, 21, false>(T, L, Lc, fc, tc, status, s);
  }
  if (T.nt == 37) {
    if (tc) return exact ? rr_as<true, 37, true>(T, L, Lc, fc, tc, status, s) : rr_as<false, 37, true>(T, L, Lc, fc, tc, status, s);
    return exact ? rr_as<true, 37, false>(T, L, Lc, fc, tc, status, s) : rr_as<false, 37, false>(T, L, Lc, fc, tc, status, s);
  }
  if (T.nt == 9) {
    if (tc) return exact ? rr_as<true, 9, true>(T, L, Lc, fc, tc, status, s) : rr_as<false, 9, true>(T, L, Lc, fc, tc, status, s);
    return exact ? rr_as<true, 9, false>(T, L, Lc, fc, tc, status, s) : rr_as<false, 9, false>(T, L, Lc, fc, tc, status, s);
  }
  if (tc) return exact ? rr_as<true, 5, true>(T, L, Lc, fc, tc, status, s) : rr_as<false, 5, true>(T, L, Lc, fc, tc, status, s);
  return exact ? rr_as<true, 5, false>(T, L, Lc, fc, tc, status, s) : rr_as<false, 5, false>(T, L, Lc, fc, tc, status, s);
}

}  // namespace nsmg
