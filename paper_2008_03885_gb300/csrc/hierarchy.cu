// Host side of the library: level layout, stencil calculus for the coarse
// operators, boundary classes, device buffers, and the cycle / solve drivers
// behind the C ABI declared in include/nsmg.h.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <new>
#include <thread>
#include <utility>
#include <vector>

#include "../../include/nsmg.h"
#include "kernels.h"
#include "tiles.h"

using namespace nsmg;

namespace {

// ---------------------------------------------------------------- stencils
// A stencil on a level's lattice: (dy, dx) -> exact dyadic weight. Keying by
// (dy, dx) makes iteration order the evaluation order of the ABI.
using Key = std::pair<int, int>;
using Stencil = std::map<Key, double>;

void put(Stencil& s, int dx, int dy, double w) {
  if (w == 0.0) return;
  s[Key(dy, dx)] += w;
  if (s[Key(dy, dx)] == 0.0) s.erase(Key(dy, dx));
}

// Own-frame offset (a, b) -> lattice offset. A rotated level's frame has
// k1 = (i - j)/2, k2 = (i + j)/2 (Sec. 4.3, Eq. G_r2), so (a, b) -> (a + b, b - a).
Key frame(int kind, int a, int b) { return kind == kRot ? Key(b - a, a + b) : Key(b, a); }

Stencil from_frame(int kind, const std::vector<std::pair<Key, double>>& st, double factor) {
  Stencil s;
  for (const auto& t : st) {
    const Key k = frame(kind, t.first.first, t.first.second);  // (dy, dx)
    put(s, k.second, k.first, t.second * factor);
  }
  return s;
}

// Own-frame stencils as ((a, b), weight).
const std::vector<std::pair<Key, double>> kFivePoint = {  // Eq. (L_h_2) times h^2
    {{0, 0}, 4.0}, {{-1, 0}, -1.0}, {{1, 0}, -1.0}, {{0, -1}, -1.0}, {{0, 1}, -1.0}};
const std::vector<std::pair<Key, double>> kFourthOrder = {  // Eq. (L_h_2d_4o) times 12 h^2
    {{0, 0}, 60.0}, {{-1, 0}, -16.0}, {{1, 0}, -16.0}, {{0, -1}, -16.0}, {{0, 1}, -16.0},
    {{-2, 0}, 1.0}, {{2, 0}, 1.0}, {{0, -2}, 1.0}, {{0, 2}, 1.0}};
const std::vector<std::pair<Key, double>> kSixthOrder = {  // Eq. (LhOrder6) times 180 h^2
    {{0, 0}, 980.0}, {{-1, 0}, -270.0}, {{1, 0}, -270.0}, {{0, -1}, -270.0}, {{0, 1}, -270.0},
    {{-2, 0}, 27.0}, {{2, 0}, 27.0}, {{0, -2}, 27.0}, {{0, 2}, 27.0},
    {{-3, 0}, -2.0}, {{3, 0}, -2.0}, {{0, -3}, -2.0}, {{0, 3}, -2.0}};
const std::vector<std::pair<Key, double>> kFirstGalerkin = {  // Eq. (L_G1) times H^2
    {{0, 0}, 3.0}, {{-1, 0}, -0.5}, {{1, 0}, -0.5}, {{0, -1}, -0.5}, {{0, 1}, -0.5},
    {{-1, -1}, -0.25}, {{1, -1}, -0.25}, {{-1, 1}, -0.25}, {{1, 1}, -0.25}};

int radius(const Stencil& s, bool x) {
  int r = 0;
  for (const auto& t : s) r = std::max(r, std::abs(x ? t.first.second : t.first.first));
  return r;
}

// ---- exact dyadic stencils (the Galerkin recursion) --------------------------------
// Galerkin coefficients are dyadic fractions whose numerators grow every level: about
// 14 bits per level with cubic transfers (past FP64's 53 from the fourth coarse level
// on) and about 3 bits per red-black level (past 53 from level 17, i.e. on grids of
// 1025^2 and more). The recursion is therefore carried exactly (value = numerator /
// 2^exp with a 256-bit signed numerator) and every level's weights are rounded once to
// FP64, as in the oracle's exact sparse products.
struct Big {
  uint64_t w[4] = {0, 0, 0, 0};  // two's complement, little-endian limbs
  static Big of(int64_t v) {
    Big b;
    const uint64_t ext = v < 0 ? ~0ull : 0ull;
    b.w[0] = (uint64_t)v;
    b.w[1] = b.w[2] = b.w[3] = ext;
    return b;
  }
  bool neg() const { return (int64_t)w[3] < 0; }
  bool zero() const { return !(w[0] | w[1] | w[2] | w[3]); }
  Big operator+(const Big& o) const {
    Big r;
    unsigned __int128 c = 0;
    for (int k = 0; k < 4; ++k) {
      c += (unsigned __int128)w[k] + o.w[k];
      r.w[k] = (uint64_t)c;
      c >>= 64;
    }
    return r;
  }
  Big negated() const {
    Big r;
    for (int k = 0; k < 4; ++k) r.w[k] = ~w[k];
    return r + of(1);
  }
  Big abs() const { return neg() ? negated() : *this; }
  // times a small integer (|m| < 2^62)
  Big times(int64_t m) const {
    const bool sn = neg() != (m < 0);
    const Big a = abs();
    const uint64_t um = (uint64_t)(m < 0 ? -m : m);
    Big r;
    unsigned __int128 c = 0;
    for (int k = 0; k < 4; ++k) {
      c += (unsigned __int128)a.w[k] * um;
      r.w[k] = (uint64_t)c;
      c >>= 64;
    }
    return sn ? r.negated() : r;
  }
  int bits() const {  // bit length of |value|
    const Big a = abs();
    for (int k = 3; k >= 0; --k)
      if (a.w[k]) return 64 * k + 64 - __builtin_clzll(a.w[k]);
    return 0;
  }
  bool even() const { return !(w[0] & 1); }
  Big half() const {  // exact division by 2 of an even value
    Big r;
    for (int k = 0; k < 4; ++k) r.w[k] = (w[k] >> 1) | (k < 3 ? (w[k + 1] << 63) : (w[3] & (1ull << 63)));
    return r;
  }
  bool bit(int i) const { return (w[i >> 6] >> (i & 63)) & 1; }
  // value * 2^-exp rounded to nearest (ties to even)
  double to_double(int exp) const {
    const Big a = abs();
    const int nb = a.bits();
    if (nb == 0) return 0.0;
    uint64_t mant;
    int shift = 0;
    if (nb <= 53) {
      mant = a.w[0];
    } else {
      shift = nb - 53;
      mant = 0;
      for (int i = 0; i < 53; ++i) mant |= (uint64_t)a.bit(shift + i) << i;
      const bool round = a.bit(shift - 1);
      bool sticky = false;
      for (int i = 0; i < shift - 1 && !sticky; ++i) sticky = a.bit(i);
      if (round && (sticky || (mant & 1))) ++mant;  // 2^53 stays exact
    }
    const double v = std::ldexp((double)mant, shift - exp);
    return neg() ? -v : v;
  }
};

struct XStencil {  // (dy, dx) -> numerator; value = numerator / 2^exp
  std::map<Key, Big> t;
  int exp = 0;
};

constexpr int kMaxExactBits = 240;

void xput(std::map<Key, Big>& s, const Key& k, const Big& v) {
  if (v.zero()) return;
  auto it = s.find(k);
  if (it == s.end()) {
    s.emplace(k, v);
    return;
  }
  it->second = it->second + v;
  if (it->second.zero()) s.erase(it);
}

// Exact copy of an integer-weighted stencil.
XStencil exact_of(const Stencil& W) {
  XStencil x;
  for (const auto& t : W) {
    const double w = t.second;
    if (w != std::floor(w) || std::fabs(w) > 1e15) return XStencil{{}, -1};  // not an integer stencil
    xput(x.t, t.first, Big::of((int64_t)w));
  }
  return x;
}

Stencil rounded(const XStencil& x) {
  Stencil s;
  for (const auto& t : x.t) s[t.first] = t.second.to_double(x.exp);
  return s;
}

// Interpolation weights from a coarse node at fine-lattice position (0, 0) to fine
// offsets (dx, dy) (Eq. transfer_r2 in the fine level's own frame; Eq. transfer_2d;
// Eq. interp_2d4o), as integers over 2^exp: ((dx, dy), tap).
struct ITaps {
  std::vector<std::pair<Key, int64_t>> t;
  int exp;
};
ITaps interp_taps(int transfer) {
  ITaps p;
  if (transfer == kStandardCubic) {  // 1D taps times 16, 2D products times 256
    const int64_t t1[7] = {-1, 0, 9, 16, 9, 0, -1};
    for (int dy = -3; dy <= 3; ++dy)
      for (int dx = -3; dx <= 3; ++dx)
        if (t1[dx + 3] && t1[dy + 3]) p.t.push_back({{dx, dy}, t1[dx + 3] * t1[dy + 3]});
    p.exp = 8;
  } else if (transfer == kRbAxisToRot) {
    p.t = {{{0, 0}, 4}, {{1, 0}, 1}, {{-1, 0}, 1}, {{0, 1}, 1}, {{0, -1}, 1}};
    p.exp = 2;
  } else if (transfer == kRbRotToAxis) {
    p.t = {{{0, 0}, 4}, {{1, 1}, 1}, {{-1, 1}, 1}, {{1, -1}, 1}, {{-1, -1}, 1}};
    p.exp = 2;
  } else {  // bilinear: (1, 2, 1) x (1, 2, 1) / 4
    const int64_t w1[3] = {1, 2, 1};
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) p.t.push_back({{dx, dy}, w1[dx + 1] * w1[dy + 1]});
    p.exp = 2;
  }
  return p;
}

// Exact Galerkin product R W P on the infinite lattice (Eq. L_G_l): the coarse stencil
// of a coarse node at the origin, with R = P^T / 2 (red-black) or P^T / 4 (standard,
// bilinear or cubic). The
// coefficients are dyadic fractions whose numerators grow every level (about 3 bits per
// red-black level, 14 per cubic level) and outgrow FP64's 53 bits on deep hierarchies,
// so the recursion is carried exactly and each level is rounded once (rounded()).
// Returns exp = -1 if a numerator would exceed kMaxExactBits.
XStencil galerkin_exact(const XStencil& W, int transfer) {
  const ITaps P = interp_taps(transfer);
  const int rexp = (transfer == kStandard || transfer == kStandardCubic) ? 2 : 1;
  const int step = transfer == kRbAxisToRot ? 1 : 2;
  int rW = 0;
  for (const auto& t : W.t) rW = std::max({rW, std::abs(t.first.first), std::abs(t.first.second)});
  const int M = (rW + 4) / step + 2;
  XStencil out;
  out.exp = W.exp + 2 * P.exp + rexp;
  for (int b = -M; b <= M; ++b)
    for (int a = -M; a <= M; ++a) {
      if (transfer == kRbAxisToRot && ((a + b) & 1)) continue;  // coarse = black points
      const int px = a * step, py = b * step;
      std::map<Key, int64_t> v;  // P e_(a,b) on the fine lattice, keyed (dy, dx)
      for (const auto& t : P.t) v[Key(py + t.first.second, px + t.first.first)] += t.second;
      Big g;
      for (const auto& r : P.t) {
        Big wv;
        for (const auto& w : W.t) {
          auto it = v.find(Key(r.first.second + w.first.first, r.first.first + w.first.second));
          if (it != v.end()) wv = wv + w.second.times(it->second);
        }
        g = g + wv.times(r.second);
      }
      if (g.bits() > kMaxExactBits) return XStencil{{}, -1};
      if (!g.zero()) out.t[Key(b, a)] = g;
    }
  // drop common factors of two
  while (out.exp > 0) {
    bool all_even = true;
    for (const auto& t : out.t) all_even = all_even && t.second.even();
    if (!all_even) break;
    for (auto& t : out.t) t.second = t.second.half();
    --out.exp;
  }
  return out;
}

// Odd-periodic reflection of t into [0, n]; sets sign and whether it lands on a boundary line.
int fold(int t, int n, double& sign, bool& bnd) {
  int m = t % (2 * n);
  if (m < 0) m += 2 * n;
  sign = m <= n ? 1.0 : -1.0;
  const int tp = m <= n ? m : 2 * n - m;
  bnd = tp == 0 || tp == n;
  return tp;
}

// Dirichlet row of node (i, j): the stencil folded by odd reflection, boundary
// columns dropped, duplicates summed, sorted by (dy, dx).
Stencil fold_row(const Stencil& st, int n, int i, int j) {
  Stencil row;
  for (const auto& t : st) {
    double si, sj;
    bool bi, bj;
    const int ti = fold(i + t.first.second, n, si, bi);
    const int tj = fold(j + t.first.first, n, sj, bj);
    if (bi || bj) continue;
    put(row, ti - i, tj - j, si * sj * t.second);
  }
  return row;
}

// The same rows from an exact stencil: the merged weights are summed exactly and
// rounded once.
Stencil fold_row_x(const XStencil& st, int n, int i, int j) {
  std::map<Key, Big> row;
  for (const auto& t : st.t) {
    double si, sj;
    bool bi, bj;
    const int ti = fold(i + t.first.second, n, si, bi);
    const int tj = fold(j + t.first.first, n, sj, bj);
    if (bi || bj) continue;
    xput(row, Key(tj - j, ti - i), si * sj < 0 ? t.second.negated() : t.second);
  }
  return rounded(XStencil{row, st.exp});
}

Stencil wrap_row_x(const XStencil& st, int n, int i, int j) {
  std::map<Key, Big> row;
  for (const auto& t : st.t) {
    int ti = (i + t.first.second) % n;
    if (ti < 0) ti += n;
    int tj = (j + t.first.first) % n;
    if (tj < 0) tj += n;
    xput(row, Key(tj - j, ti - i), t.second);
  }
  return rounded(XStencil{row, st.exp});
}

// Periodic row of node (i, j): offsets wrapped modulo n into [0, n), duplicates
// summed, sorted by (dy, dx) of the wrapped offset (the column order).
Stencil wrap_row(const Stencil& st, int n, int i, int j) {
  Stencil row;
  for (const auto& t : st) {
    int ti = (i + t.first.second) % n;
    if (ti < 0) ti += n;
    int tj = (j + t.first.first) % n;
    if (tj < 0) tj += n;
    put(row, ti - i, tj - j, t.second);
  }
  return row;
}

struct LevelShape {
  int kind, n;
  double hh;  // (h_l / h_0)^2
};

std::vector<LevelShape> level_shapes(int N, int coarsening, int n_min, int max_levels) {
  std::vector<LevelShape> s{{kAxis, N, 1.0}};
  for (;;) {
    const LevelShape c = s.back();
    if (max_levels > 0 && (int)s.size() >= max_levels) break;
    if (c.kind == kAxis && c.n <= n_min) break;
    // variable coarsening (Sec. 4.4): red-black for levels 1 and 2, standard below
    const bool rb = coarsening == MG_COARSEN_REDBLACK || (coarsening == MG_COARSEN_VARIABLE && s.size() < 3);
    if (rb)
      s.push_back(c.kind == kAxis ? LevelShape{kRot, c.n, 2.0 * c.hh} : LevelShape{kAxis, c.n / 2, 2.0 * c.hh});
    else
      s.push_back({kAxis, c.n / 2, 4.0 * c.hh});
  }
  return s;
}

// Transfer between level l (fine) and l + 1 (transfer_order 4: cubic, standard
// coarsening only).
int transfer_of(int coarsening, int l, int fine_kind, int transfer_order) {
  if (coarsening == MG_COARSEN_STANDARD) return transfer_order == 4 ? kStandardCubic : kStandard;
  if (coarsening == MG_COARSEN_VARIABLE && l >= 2) return kStandard;
  return fine_kind == kAxis ? kRbAxisToRot : kRbRotToAxis;
}

// Host-side build of one level's operator description (both precisions).
struct HostLevel {
  LevelShape shape;
  int per = 0;  // periodic level: unknowns 0 <= i, j < n, stencils wrap
  int boundary_data = 0;  // level 0 with Dirichlet data g: fast stencils read the boundary
  int exact = 0;  // W is the rounding of the exact stencil Wx (boundary rows from Wx)
  XStencil Wx;
  int rows, cols, pitch;
  Stencil W;  // exact weights
  double s;   // scale: coefficient = fl(w * s)
  // boundary classes
  int small, clsw, ncls;
  std::vector<int2> cls;
  std::vector<double> cls_wd;
  std::vector<int32_t> tdx, tdy;
  std::vector<double> tc;
  double wd_fast = 0.0;
  int rx = 0, ry = 0;
  std::vector<double> c;  // fast coefficients, in evaluation order (group_terms)
  std::vector<int> dxs, dys;
  std::vector<uint8_t> gstart;  // 1: the fast term starts a group
  std::vector<uint8_t> tstart;  // class terms: 1 starts a group
  int64_t unknowns = 0;
};

int storage_cols(int kind, int n) { return kind == kAxis ? n + 1 : n / 2 + 1; }
int round_pitch(int cols) { return (cols + 31) / 32 * 32; }

// Evaluation order of an operator row (terms given in (dy, dx), i.e. storage column,
// order): the terms are split into groups of equal coefficient, the groups ordered by
// their first term and each group's terms kept in column order; `start` flags the first
// term of every group. The row is then evaluated as sum_g c_g * (x_g1 + x_g2 + ...).
void group_terms(std::vector<int>& dx, std::vector<int>& dy, std::vector<double>& c, std::vector<uint8_t>& start) {
  const size_t m = c.size();
  std::vector<int> grp(m, -1), first;  // group of each term; first term of each group
  for (size_t k = 0; k < m; ++k) {
    for (size_t g = 0; g < first.size() && grp[k] < 0; ++g)
      if (c[first[g]] == c[k]) grp[k] = (int)g;
    if (grp[k] < 0) {
      grp[k] = (int)first.size();
      first.push_back((int)k);
    }
  }
  std::vector<int> dx2, dy2;
  std::vector<double> c2;
  start.clear();
  for (size_t g = 0; g < first.size(); ++g)
    for (size_t k = 0; k < m; ++k)
      if (grp[k] == (int)g) {
        start.push_back((int)k == first[g] ? 1 : 0);
        dx2.push_back(dx[k]);
        dy2.push_back(dy[k]);
        c2.push_back(c[k]);
      }
  dx.swap(dx2);
  dy.swap(dy2);
  c.swap(c2);
}

void build_classes(HostLevel& L, double omega) {
  const int n = L.shape.n;
  // Fast nodes use the plain stencil. With homogeneous Dirichlet data a fast stencil must
  // not reach a boundary line either: the operator's rows drop boundary columns, and a
  // term of value 0 kept in a row would change its groups of equal coefficient (the
  // evaluation order). So the fast range starts one node further in (radius + 1);
  // periodic rows wrap, and with Dirichlet data g the stencil reads the boundary values.
  const int ext = (L.per || L.boundary_data) ? 0 : 1;
  L.rx = radius(L.W, true) + ext;
  L.ry = radius(L.W, false) + ext;
  for (const auto& t : L.W) {
    L.c.push_back(t.second * L.s);
    L.dxs.push_back(t.first.second);
    L.dys.push_back(t.first.first);
  }
  group_terms(L.dxs, L.dys, L.c, L.gstart);
  L.wd_fast = omega / (L.W.at(Key(0, 0)) * L.s);
  const int R = std::max(L.rx, L.ry);
  const int e = n - L.per;  // last lattice index a fast stencil may reach
  const int lo = 1 - L.per;  // first unknown index
  L.small = (n <= 4 * R + 4) ? 1 : 0;
  L.clsw = L.small ? n + 1 : 2 * L.rx + 1;
  const int clsh = L.small ? n + 1 : 2 * L.ry + 1;
  L.ncls = L.clsw * clsh;
  L.cls.assign(L.ncls, make_int2(0, 0));
  L.cls_wd.assign(L.ncls, 0.0);
  auto rep = [&](int c, int r) -> int {  // representative coordinate of class c
    if (c < r) return c;
    if (c > r) return e - (2 * r - c);
    return n / 2;
  };
  for (int cy = 0; cy < clsh; ++cy)
    for (int cx = 0; cx < L.clsw; ++cx) {
      const int i = L.small ? cx : rep(cx, L.rx);
      const int j = L.small ? cy : rep(cy, L.ry);
      const int k = cy * L.clsw + cx;
      if (i < lo || i >= n || j < lo || j >= n) continue;
      if (L.small && L.shape.kind == kRot && ((i + j) & 1)) continue;
      const Stencil row = L.exact ? (L.per ? wrap_row_x(L.Wx, n, i, j) : fold_row_x(L.Wx, n, i, j))
                                  : (L.per ? wrap_row(L.W, n, i, j) : fold_row(L.W, n, i, j));
      L.cls[k] = make_int2((int)L.tdx.size(), (int)row.size());
      double diag = 0.0;
      std::vector<int> rdx, rdy;
      std::vector<double> rc;
      std::vector<uint8_t> rst;
      for (const auto& t : row) {
        rdx.push_back(t.first.second);
        rdy.push_back(t.first.first);
        rc.push_back(t.second * L.s);
        if (t.first.first == 0 && t.first.second == 0) diag = t.second * L.s;
      }
      group_terms(rdx, rdy, rc, rst);
      L.tdx.insert(L.tdx.end(), rdx.begin(), rdx.end());
      L.tdy.insert(L.tdy.end(), rdy.begin(), rdy.end());
      L.tc.insert(L.tc.end(), rc.begin(), rc.end());
      L.tstart.insert(L.tstart.end(), rst.begin(), rst.end());
      L.cls_wd[k] = omega / diag;
    }
}

template <typename T>
LevelDev<T> to_dev(const HostLevel& L) {
  LevelDev<T> d;
  std::memset(&d, 0, sizeof(d));
  d.kind = L.shape.kind;
  d.n = L.shape.n;
  d.rows = L.rows;
  d.cols = L.cols;
  d.pitch = L.pitch;
  d.nt = (int)L.c.size();
  d.rx = L.rx;
  d.ry = L.ry;
  d.small = L.small;
  d.clsw = L.clsw;
  d.per = L.per;
  d.lo = 1 - L.per;
  d.fxe = L.shape.n - L.per - L.rx;
  d.fye = L.shape.n - L.per - L.ry;
  d.wd = (T)L.wd_fast;
  for (int k = 0; k < d.nt; ++k) {
    d.c[k] = (T)L.c[k];
    const int dx = L.dxs[k], dy = L.dys[k];
    if (L.shape.kind == kRot) {
      // column of (i + dx) >> 1 relative to i >> 1 for i even / odd
      d.sdx[0][k] = dx >= 0 ? dx / 2 : -((-dx + 1) / 2);
      d.sdx[1][k] = (dx + 1) >= 0 ? (dx + 1) / 2 : -((-(dx + 1) + 1) / 2);
    } else {
      d.sdx[0][k] = d.sdx[1][k] = dx;
    }
    d.sdy[k] = dy;
    d.delta[0][k] = dy * L.pitch + d.sdx[0][k];
    d.delta[1][k] = dy * L.pitch + d.sdx[1][k];
    if (L.gstart[k]) d.gmask[k >> 5] |= 1u << (k & 31);
  }
  return d;
}

}  // namespace

// ---------------------------------------------------------------- handle
// Device hierarchy in one precision.
template <typename T>
struct Hier {
  std::vector<LevelPair<T>> L;
  std::vector<T*> u, t, f, d;  // FP64 level 0: u and f are the caller's
  int64_t coarsest_idx = 0;
  T coarsest_a = T(1);
  int coarsest_zero = 0;  // periodic: the coarsest single node's zero-mean solution is 0
  DenseCoarse<T> dense{};  // m > 0: the coarsest level has m > 1 unknowns (dense solve)
  // small-level tail (one thread block runs the sub-cycle from tail_level down)
  int tail_level = -1;
  TailDesc<T>* d_tail = nullptr;
  int4* d_prog = nullptr;  // program for a sub-cycle with zero initial guess
  int nops = 0;
  int tail_ctas = 1;       // CTAs in the tail's thread-block cluster
  int tail_smem = 0;       // > 0: the tail's levels live in shared memory (elements)
  std::vector<TileLevel> tiles;  // FP32 levels: TMA tile kernels (tiles.h) where eligible
};

struct mg_handle {
  int N = 0, order = 2, coarsening = 1, coarse_op = 1;
  double length = 1.0;  // side of the square domain
  mg_options opt;
  std::vector<HostLevel> host;
  std::vector<int> transfer;
  Hier<double> h64;
  Hier<float> h32;  // mixed precision: inner cycles (level 0 = scaled residual / correction)
  double* partial = nullptr;
  double* scalar = nullptr;      // device
  double* hscalar = nullptr;     // pinned host
  std::vector<void*> allocs;     // every cudaMalloc / cudaMallocHost to free
  std::vector<void*> host_allocs;
  int nblocks0 = 0;
  double ir_scale = 0.0;  // mixed precision: scale of the next refinement residual (0 = unset)
  // CUDA graphs of the cycle: the FP64 cycle on the caller's (u, f), and the FP32
  // inner cycles of the mixed-precision path (internal buffers only)
  struct GraphEntry {
    const void* u = nullptr;
    const void* f = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;
  };
  GraphEntry g_cycle64, g_cycle64r, g_inner32;  // g_cycle64r: level 0's first red half-sweep done
  cudaStream_t priv = nullptr;  // used when the caller passes the legacy default stream
  double* host_u = nullptr;     // mg_solve_host: device copies of the caller's u and f
  double* host_f = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // instrumentation
  int64_t launches = 0, cycles = 0;
  int timing = 0;  // 1: finest-level kernels, 2: every level (class + 5 * level)
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[MG_KERNEL_CLASSES * (kTailMaxLevels + 1)];
  size_t ev_used[MG_KERNEL_CLASSES * (kTailMaxLevels + 1)] = {};
};

template <typename T>
Hier<T>& hier(mg_handle* h);
template <>
Hier<double>& hier<double>(mg_handle* h) { return h->h64; }
template <>
Hier<float>& hier<float>(mg_handle* h) { return h->h32; }

namespace {

#define CK(x)                                 \
  do {                                        \
    if ((x) != cudaSuccess) return MG_ERR_CUDA; \
  } while (0)

// Launch `nk` kernels through `expr`, counting them.
#define LAUNCH(h, nk, expr)                       \
  do {                                            \
    (h)->launches += (nk);                        \
    if ((expr) != cudaSuccess) return MG_ERR_CUDA; \
  } while (0)

// CUDA-event bracket around finest-level launches of one kernel class.
struct Bracket {
  mg_handle* h;
  int cls;
  cudaStream_t s;
  bool on;
  Bracket(mg_handle* h_, int level, int cls_, cudaStream_t s_)
      : h(h_), cls(cls_ + (h_->timing == 2 ? MG_KERNEL_CLASSES * level : 0)), s(s_),
        on(h_->timing == 2 ? level <= kTailMaxLevels : (h_->timing != 0 && level == 0)) {
    if (!on) return;
    auto& v = h->ev[cls];
    if (h->ev_used[cls] == v.size()) {
      cudaEvent_t a, b;
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      v.push_back({a, b});
    }
    cudaEventRecord(v[h->ev_used[cls]].first, s);
  }
  ~Bracket() {
    if (!on) return;
    cudaEventRecord(h->ev[cls][h->ev_used[cls]].second, s);
    ++h->ev_used[cls];
  }
};

bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// Lattice size of the coarsest axis level: n_min (Dirichlet: one interior unknown at
// n = 2), or 1 for periodic hierarchies (a single node).
int coarsest_n(const mg_options& o) { return o.boundary == MG_BOUNDARY_PERIODIC ? 1 : o.n_min; }

mg_status validate(const mg_grid* grid, int order, int coarsening, int coarse_op, const mg_options& o) {
  if (!grid || !pow2(grid->n) || grid->n < 4 || grid->n > 16384) return MG_ERR_INVALID;
  if (!(grid->length >= 0.0) || !std::isfinite(grid->length)) return MG_ERR_INVALID;
  if (order != 2 && order != 4 && order != 6) return MG_ERR_INVALID;
  if (coarsening != MG_COARSEN_STANDARD && coarsening != MG_COARSEN_REDBLACK && coarsening != MG_COARSEN_VARIABLE)
    return MG_ERR_INVALID;
  if (coarse_op < MG_OP_NONGALERKIN || coarse_op > MG_OP_NONGALERKIN_HIGH) return MG_ERR_INVALID;
  if (!(o.omega > 0.0 && o.omega < 2.0) || o.nu1 < 0 || o.nu2 < 0 || o.nu1 + o.nu2 < 1 ||
      o.gamma < 1 || o.gamma > 3 || (o.smoother != MG_SMOOTH_REDBLACK && o.smoother != MG_SMOOTH_JACOBI))
    return MG_ERR_INVALID;
  if (o.precision != MG_PREC_FP64 && o.precision != MG_PREC_MIXED_FP32) return MG_ERR_INVALID;
  if (o.precision == MG_PREC_MIXED_FP32 && (o.inner_cycles < 1 || o.inner_cycles > 64)) return MG_ERR_INVALID;
  if (o.tail_ctas < 0 || o.tail_ctas > 16) return MG_ERR_INVALID;
  if (o.sweep_kernel < 0 || o.sweep_kernel > 2) return MG_ERR_INVALID;
  if (o.bf16_levels < 0 || o.bf16_levels > 4) return MG_ERR_INVALID;
  if (o.bf16_levels > 0 && (o.precision != MG_PREC_MIXED_FP32 || o.sweep_kernel == 2)) return MG_ERR_UNSUPPORTED;
  if (o.boundary != MG_BOUNDARY_DIRICHLET && o.boundary != MG_BOUNDARY_PERIODIC) return MG_ERR_INVALID;
  if (o.transfer_order != 2 && o.transfer_order != 4) return MG_ERR_INVALID;
  if ((o.dev_alloc == nullptr) != (o.dev_free == nullptr)) return MG_ERR_INVALID;
  if (o.dirichlet_data != 0 && o.dirichlet_data != 1) return MG_ERR_INVALID;
  if (o.dirichlet_data == 1 && (order != 2 || o.boundary != MG_BOUNDARY_DIRICHLET)) return MG_ERR_UNSUPPORTED;
  if (o.transfer_order == 4 && coarsening != MG_COARSEN_STANDARD) return MG_ERR_UNSUPPORTED;
  if (o.boundary == MG_BOUNDARY_PERIODIC && o.sweep_kernel == 2) return MG_ERR_UNSUPPORTED;
  if (!pow2(o.n_min) || o.n_min < 2 || o.max_levels < 0) return MG_ERR_INVALID;
  // at least two levels; a coarsest level with several unknowns takes the dense solve,
  // which is built for Dirichlet boundaries
  if (o.n_min > grid->n / 2 || o.max_levels == 1) return MG_ERR_UNSUPPORTED;
  if (o.boundary == MG_BOUNDARY_PERIODIC && (o.n_min != 2 || o.max_levels != 0)) return MG_ERR_UNSUPPORTED;
  return MG_OK;
}

// Level operators for the chosen coarse-operator family (Sec. 2.3 notation).
// Returns false if an exact Galerkin recursion outgrows its integer width.
bool build_operators(mg_handle* h, const std::vector<LevelShape>& shapes) {
  const double hf = h->length / h->N;
  const double s2 = 1.0 / (hf * hf);         // operators derived from L_h^(2)
  const double s4 = 1.0 / (12.0 * hf * hf);  // operators derived from L_h^(4)
  const int nl = (int)shapes.size();
  h->host.resize(nl);
  for (int l = 0; l < nl; ++l) h->host[l].shape = shapes[l];
  HostLevel& L0 = h->host[0];
  L0.boundary_data = h->opt.dirichlet_data;
  Stencil base;
  double base_s;
  if (h->order == 2) {
    L0.W = from_frame(kAxis, kFivePoint, 1.0);
    L0.s = s2;
    base = L0.W;
    base_s = s2;
  } else {
    // fourth or sixth order: coarse levels from L_h^(2) unless "true high"
    const double s6 = 1.0 / (180.0 * hf * hf);
    L0.W = from_frame(kAxis, h->order == 4 ? kFourthOrder : kSixthOrder, 1.0);
    L0.s = h->order == 4 ? s4 : s6;
    if (h->coarse_op == MG_OP_GALERKIN_TRUE_HIGH) {
      base = L0.W;
      base_s = L0.s;
    } else {
      base = from_frame(kAxis, kFivePoint, 1.0);
      base_s = s2;
    }
  }
  const int op = h->coarse_op;
  // the Galerkin recursion in exact arithmetic, each level rounded once (see XStencil)
  XStencil galx = exact_of(base);
  if (galx.exp < 0) return false;
  for (int l = 1; l < nl; ++l) {
    HostLevel& L = h->host[l];
    const bool galerkin_level =
        op == MG_OP_GALERKIN || op == MG_OP_GALERKIN_TRUE_HIGH || (op == MG_OP_GALERKIN_GN && l == 1);
    if (galerkin_level) {
      galx = galerkin_exact(galx, transfer_of(h->coarsening, l - 1, shapes[l - 1].kind, h->opt.transfer_order));
      if (galx.exp < 0) return false;
    }
    if (galerkin_level) {
      L.W = rounded(galx);
      L.Wx = galx;
      L.exact = 1;
      L.s = base_s;
    } else if (op == MG_OP_GALERKIN_G1) {
      L.W = from_frame(L.shape.kind, kFirstGalerkin, 1.0 / L.shape.hh);
      L.s = s2;
    } else if (op == MG_OP_NONGALERKIN_HIGH && h->order > 2) {
      // the fine operator's stencil with spacing H (nG^(4), Eq. L_H_4n_2d; nG^(6))
      L.W = from_frame(L.shape.kind, h->order == 4 ? kFourthOrder : kSixthOrder, 1.0 / L.shape.hh);
      L.s = L0.s;
    } else {
      L.W = from_frame(L.shape.kind, kFivePoint, 1.0 / L.shape.hh);
      L.s = s2;
    }
  }
  for (int l = 0; l < nl; ++l) {
    HostLevel& L = h->host[l];
    L.per = h->opt.boundary == MG_BOUNDARY_PERIODIC ? 1 : 0;
    L.rows = L.shape.n + 1;
    L.cols = storage_cols(L.shape.kind, L.shape.n);
    L.pitch = l == 0 ? L.cols : round_pitch(L.cols);
    if (L.per) {
      const int64_t m = L.shape.n;  // nodes 0 .. n-1; n even on rotated levels
      L.unknowns = L.shape.kind == kAxis ? m * m : m * m / 2;
    } else {
      const int64_t m = L.shape.n - 1;
      L.unknowns = L.shape.kind == kAxis ? m * m : (m * m + 1) / 2;
    }
    build_classes(L, h->opt.omega);
  }
  return true;
}

size_t level_bytes(const HostLevel& L, size_t elem) { return (size_t)L.rows * L.pitch * elem; }

// Storage description of level l in precision T: the FP64 finest level keeps the
// caller's (N+1)-element rows; every other level, and the FP32 finest level of the
// mixed-precision path, pads its rows to a multiple of 32 elements (so that rows start
// on 16-byte boundaries, as TMA tile loads require).
template <typename T>
HostLevel storage_of(const HostLevel& L, int l) {
  HostLevel S = L;
  if (l == 0 && sizeof(T) == 4) S.pitch = round_pitch(L.cols);
  return S;
}

// Largest coarsest system solved by the dense factor (2 x m^2 values per precision).
constexpr int kDenseMaxUnknowns = 1024;

// Inverse Cholesky factor G = L^-1 of the coarsest operator (level C, Dirichlet), in
// the unknown order row-major (j, then i), every product and sum rounded separately:
// Cholesky by columns j (s = A_jj - L_j0 L_j0 - ... with k ascending, L_jj = sqrt(s),
// r_j = 1 / L_jj, L_ij = (A_ij - L_i0 L_j0 - ...) r_j), then G by rows i (G_ii = r_i,
// G_ic = -((L_ic G_cc + L_i,c+1 G_c+1,c + ... + L_i,i-1 G_i-1,c) r_i)). A's entries
// are the level's coefficients fl(w s), as in its stencil kernels. Returns false if
// the operator is not positive definite.
bool dense_factor(const HostLevel& C, std::vector<double>& G, std::vector<int2>& ij) {
  const int n = C.shape.n;
  std::vector<int> index((size_t)(n + 1) * (n + 1), -1);
  ij.clear();
  for (int j = 1; j < n; ++j)
    for (int i = 1; i < n; ++i) {
      if (C.shape.kind == kRot && ((i + j) & 1)) continue;
      index[(size_t)j * (n + 1) + i] = (int)ij.size();
      ij.push_back(make_int2(i, j));
    }
  const size_t m = ij.size();
  std::vector<double> A(m * m, 0.0);
  for (size_t p = 0; p < m; ++p) {
    const int i = ij[p].x, j = ij[p].y;
    const Stencil row = C.exact ? fold_row_x(C.Wx, n, i, j) : fold_row(C.W, n, i, j);
    for (const auto& t : row) {
      const int q = index[(size_t)(j + t.first.first) * (n + 1) + (i + t.first.second)];
      if (q < 0) return false;
      A[p * m + q] = t.second * C.s;
    }
  }
  std::vector<double> L(m * m, 0.0), r(m);
  for (size_t j = 0; j < m; ++j) {
    double sd = A[j * m + j];
    for (size_t k = 0; k < j; ++k) sd = sd - L[j * m + k] * L[j * m + k];
    if (!(sd > 0.0)) return false;
    L[j * m + j] = std::sqrt(sd);
    r[j] = 1.0 / L[j * m + j];
    for (size_t i = j + 1; i < m; ++i) {
      double t = A[i * m + j];
      for (size_t k = 0; k < j; ++k) t = t - L[i * m + k] * L[j * m + k];
      L[i * m + j] = t * r[j];
    }
  }
  G.assign(m * m, 0.0);
  std::vector<double> acc(m);
  for (size_t i = 0; i < m; ++i) {
    G[i * m + i] = r[i];
    for (size_t k = 0; k < i; ++k) {
      const double lik = L[i * m + k];
      acc[k] = lik * G[k * m + k];  // the first product of column k's sum
      for (size_t c = 0; c < k; ++c) acc[c] = acc[c] + lik * G[k * m + c];
    }
    for (size_t c = 0; c < i; ++c) G[i * m + c] = -(acc[c] * r[i]);
  }
  return true;
}

mg_status device_alloc(mg_handle* h, void** p, size_t bytes) {
  if (bytes == 0) bytes = 256;
  if (h->opt.dev_alloc) {  // caller's allocator
    *p = h->opt.dev_alloc(bytes, h->opt.alloc_ctx);
    if (!*p) return MG_ERR_OOM;
  } else {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA;
    }
  }
  h->allocs.push_back(*p);
  if (cudaMemsetAsync(*p, 0, bytes, h->priv) != cudaSuccess) return MG_ERR_CUDA;
  return MG_OK;
}

// Device copies of the dense coarsest factor in precision T (FP32: G rounded once).
template <typename T>
mg_status upload_dense(mg_handle* h, const std::vector<double>& G, const std::vector<int2>& ij, DenseCoarse<T>& D) {
  const size_t m = ij.size();
  std::vector<T> ga(m * m), gb(m * m);
  for (size_t k = 0; k < m; ++k)
    for (size_t i = 0; i < m; ++i) {
      ga[k * m + i] = (T)G[i * m + k];
      gb[k * m + i] = (T)G[k * m + i];
    }
  T *dga, *dgb;
  int2* dij;
  mg_status st;
  if ((st = device_alloc(h, (void**)&dga, m * m * sizeof(T))) != MG_OK) return st;
  if ((st = device_alloc(h, (void**)&dgb, m * m * sizeof(T))) != MG_OK) return st;
  if ((st = device_alloc(h, (void**)&dij, m * sizeof(int2))) != MG_OK) return st;
  CK(cudaMemcpyAsync(dga, ga.data(), m * m * sizeof(T), cudaMemcpyHostToDevice, h->priv));
  CK(cudaMemcpyAsync(dgb, gb.data(), m * m * sizeof(T), cudaMemcpyHostToDevice, h->priv));
  CK(cudaMemcpyAsync(dij, ij.data(), m * sizeof(int2), cudaMemcpyHostToDevice, h->priv));
  CK(cudaStreamSynchronize(h->priv));  // the host vectors go out of scope
  D.ga = dga;
  D.gb = dgb;
  D.ij = dij;
  D.m = (int)m;
  return MG_OK;
}

template <typename T>
mg_status upload_level(mg_handle* h, const HostLevel& L, LevelPair<T>& P, int bf16 = 0) {
  P.h = to_dev<T>(L);
  P.h.bf16 = bf16;
  int2* cls;
  T* cwd;
  ClassTerm<T>* terms;
  mg_status st;
  const size_t nt = std::max<size_t>(L.tdx.size(), 1);
  if ((st = device_alloc(h, (void**)&cls, L.cls.size() * sizeof(int2))) != MG_OK) return st;
  if ((st = device_alloc(h, (void**)&cwd, L.cls_wd.size() * sizeof(T))) != MG_OK) return st;
  if ((st = device_alloc(h, (void**)&terms, nt * sizeof(ClassTerm<T>))) != MG_OK) return st;
  std::vector<T> wd(L.cls_wd.begin(), L.cls_wd.end());
  std::vector<ClassTerm<T>> tt(L.tdx.size());
  for (size_t k = 0; k < tt.size(); ++k) {
    std::memset(&tt[k], 0, sizeof(tt[k]));
    tt[k].c = (T)L.tc[k];
    tt[k].dx = L.tdx[k] + (L.tstart[k] ? kTermStart : 0);
    tt[k].dy = L.tdy[k];
  }
  CK(cudaMemcpyAsync(cls, L.cls.data(), L.cls.size() * sizeof(int2), cudaMemcpyHostToDevice, h->priv));
  CK(cudaMemcpyAsync(cwd, wd.data(), wd.size() * sizeof(T), cudaMemcpyHostToDevice, h->priv));
  if (!tt.empty())
    CK(cudaMemcpyAsync(terms, tt.data(), tt.size() * sizeof(ClassTerm<T>), cudaMemcpyHostToDevice, h->priv));
  P.h.cls = cls;
  P.h.cls_wd = cwd;
  P.h.terms = terms;
  if ((st = device_alloc(h, (void**)&P.d, sizeof(LevelDev<T>))) != MG_OK) return st;
  CK(cudaMemcpyAsync(P.d, &P.h, sizeof(LevelDev<T>), cudaMemcpyHostToDevice, h->priv));
  return MG_OK;
}

void free_all(mg_handle* h) {
  for (auto* g : {&h->g_cycle64, &h->g_cycle64r, &h->g_inner32})
    if (g->exec) cudaGraphExecDestroy(g->exec);
  if (h->priv) cudaStreamDestroy(h->priv);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  for (auto& v : h->ev)
    for (auto& e : v) {
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
  if (h->opt.dev_free) {
    // the caller's allocator may hand the memory out again at once: wait for every stream
    if (!h->allocs.empty()) cudaDeviceSynchronize();
    for (void* p : h->allocs) h->opt.dev_free(p, h->opt.alloc_ctx);
  } else {
    for (void* p : h->allocs) cudaFree(p);
  }
  for (void* p : h->host_allocs) cudaFreeHost(p);
  h->allocs.clear();
  h->host_allocs.clear();
}

// Coarse-level cycles per visit of level l: gamma 1 (V), 2 (W), or 3 = "Wn" (Sec. 4.4):
// two on levels 0 and 1, one below.
int gamma_at(const mg_handle* h, int l) {
  if (h->opt.gamma == 3) return l <= 1 ? 2 : 1;
  return h->opt.gamma;
}

// ---------------------------------------------------------------- cycle
struct Ctx {
  mg_handle* h;
  cudaStream_t s;
  bool exact;
};

// The handle's device status word (bits set by kernels whose bounded waits gave up),
// kept next to the norm scalar so that one copy reads both.
int* status_word(mg_handle* h) { return reinterpret_cast<int*>(h->scalar + 1); }

// The FP32 view of a level, for the tile-kernel calls (reached only when T = float:
// tile_at<double> is always null).
template <typename T>
const LevelPair<float>& f32(const LevelPair<T>& L) {
  return reinterpret_cast<const LevelPair<float>&>(L);
}

// Tile kernels of FP32 level l (tiles.h), or null: FP64 levels and levels that keep the
// per-step kernels.
template <typename T>
const TileLevel* tile_at(const mg_handle* h, int l);
template <>
const TileLevel* tile_at<double>(const mg_handle*, int) { return nullptr; }
template <>
const TileLevel* tile_at<float>(const mg_handle* h, int l) {
  return l < (int)h->h32.tiles.size() && h->h32.tiles[l].on ? &h->h32.tiles[l] : nullptr;
}

// Work of an API call runs on the caller's stream, or -- for the legacy default
// stream, which cannot be captured into a graph -- on the handle's own stream,
// ordered after the caller's earlier work and before its later work by events.
struct StreamScope {
  mg_handle* h;
  cudaStream_t user, s;
  StreamScope(mg_handle* h_, void* stream) : h(h_), user((cudaStream_t)stream), s((cudaStream_t)stream) {
    if (user || !h->priv) return;
    cudaEventRecord(h->ev_in, user);
    cudaStreamWaitEvent(h->priv, h->ev_in, 0);
    s = h->priv;
  }
  ~StreamScope() {
    if (s == user) return;
    cudaEventRecord(h->ev_out, s);
    cudaStreamWaitEvent(user, h->ev_out, 0);
  }
};

// Run `body` (a sequence of launches on c.s) through a cached CUDA graph keyed by
// (u, f). Launched eagerly when timing is on (events need eager launches) or when
// the caller is already capturing the stream (the launches join the caller's graph).
template <typename Body>
mg_status run_graph(const Ctx& c, mg_handle::GraphEntry& g, const void* u, const void* f, Body body) {
  mg_handle* h = c.h;
  if (h->timing || c.s == nullptr) return body();
  if (g.exec && g.u == u && g.f == f) {
    CK(cudaGraphLaunch(g.exec, c.s));
    h->launches += g.kernels;
    return MG_OK;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(c.s, &cs));
  if (cs != cudaStreamCaptureStatusNone) return body();
  const int64_t before = h->launches;
  CK(cudaStreamBeginCapture(c.s, cudaStreamCaptureModeThreadLocal));
  const mg_status st = body();
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c.s, &graph);
  if (st != MG_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    if (st != MG_OK) return st;
    // The capture was invalidated (e.g. by another thread's synchronising call):
    // nothing of it ran, so launch the same work eagerly.
    cudaGetLastError();
    h->launches = before;
    return body();
  }
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    cudaGetLastError();
    h->launches = before;
    return body();
  }
  if (g.exec) cudaGraphExecDestroy(g.exec);
  g.u = u;
  g.f = f;
  g.exec = exec;
  g.kernels = h->launches - before;
  h->launches = before + g.kernels;
  CK(cudaGraphLaunch(exec, c.s));
  return MG_OK;
}

// Red-black sweeps through the shared-memory tile kernel (one launch per sweep)?
// Auto uses the two half-sweep kernels: on GB300 they are faster in both precisions
// (measured: FP32 level-0 sweep 2 x 87 us vs 180 us; FP64 2 x 336 us vs 1080 us).
template <typename T>
bool fused_sweeps(const mg_handle* h) {
  if (h->opt.smoother != MG_SMOOTH_REDBLACK) return false;
  return h->opt.sweep_kernel == 2;
}

// One smoothing sweep in place on U (the handle's t[l] is the scratch buffer).
template <typename T>
mg_status smooth(const Ctx& c, int l, T* U, const T* F) {
  mg_handle* h = c.h;
  Hier<T>& H = hier<T>(h);
  T* Tb = H.t[l];
  const auto& L = H.L[l];
  if (fused_sweeps<T>(h)) {
    {
      Bracket b(h, l, MG_KERNEL_SMOOTH, c.s);
      LAUNCH(h, 1, launch_sweep_fused<T>(L, c.exact, U, F, Tb, c.s));
    }
    CK(cudaMemcpyAsync(U, Tb, level_bytes(storage_of<T>(h->host[l], l), sizeof(T)), cudaMemcpyDeviceToDevice, c.s));
  } else if (h->opt.smoother == MG_SMOOTH_REDBLACK) {
    {
      Bracket b(h, l, MG_KERNEL_SMOOTH, c.s);
      LAUNCH(h, 1, launch_half_sweep<T>(L, c.exact, U, F, Tb, 1, c.s));
    }
    Bracket b(h, l, MG_KERNEL_SMOOTH, c.s);
    LAUNCH(h, 1, launch_half_sweep<T>(L, c.exact, Tb, F, U, 0, c.s));
  } else {
    Bracket b(h, l, MG_KERNEL_SMOOTH, c.s);
    LAUNCH(h, 1, launch_jacobi<T>(L, c.exact, U, F, Tb, c.s));
    CK(cudaMemcpyAsync(U, Tb, level_bytes(storage_of<T>(h->host[l], l), sizeof(T)), cudaMemcpyDeviceToDevice, c.s));
  }
  return MG_OK;
}

// Smoothing sweep inside a cycle: tile-kernel sweeps alternate between *cur and the
// level's t buffer (out of place, no copy back); other sweeps stay in *cur.
template <typename T>
mg_status cycle_sweep(const Ctx& c, int l, T*& cur, T*& oth, const T* F) {
  mg_handle* h = c.h;
  if (!fused_sweeps<T>(h)) return smooth<T>(c, l, cur, F);
  {
    Bracket b(h, l, MG_KERNEL_SMOOTH, c.s);
    LAUNCH(h, 1, launch_sweep_fused<T>(hier<T>(h).L[l], c.exact, cur, F, oth, c.s));
  }
  std::swap(cur, oth);
  return MG_OK;
}

// Whether level l of precision T starts its cycles with the fused tile presmooth
// (tiles.h): its first red half-sweep is then not done by the kernel before it.
template <typename T>
bool tile_presmooth(const mg_handle* h, int l) {
  const TileLevel* tl = tile_at<T>(h, l);
  return tl && tl->nu1 == h->opt.nu1 && h->opt.smoother == MG_SMOOTH_REDBLACK;
}

// red_done: the first half-sweep (red) of the first pre-smoothing sweep already left its
// result in the level's t buffer (the residual-norm kernel did it); start with black.
template <typename T>
mg_status cycle_level(const Ctx& c, int l, T* U, const T* F, bool zero_init, bool red_done = false) {
  mg_handle* h = c.h;
  Hier<T>& H = hier<T>(h);
  const int lmax = (int)h->host.size() - 1;
  mg_status st;
  if (l == H.tail_level) {
    // the program starts with the zeroing op; skip it to continue from U
    const int4* prog = zero_init ? H.d_prog : H.d_prog + 1;
    const int nops = zero_init ? H.nops : H.nops - 1;
    Bracket b(h, l, MG_KERNEL_SMOOTH, c.s);
    if (H.tail_smem > 0)
      LAUNCH(h, 1, launch_tail_smem<T>(H.d_tail, H.tail_smem, (int)h->host.size() - H.tail_level, prog, nops,
                                       c.exact, c.s));
    else LAUNCH(h, 1, launch_tail<T>(H.tail_ctas, H.d_tail, prog, nops, c.exact, c.s));
    return MG_OK;
  }
  // FP32 levels with tile kernels: nu1 sweeps from u = 0 in one kernel, the residual
  // fused with the red-black restriction, and post-smoothing sweeps as one kernel each
  // (ping-pong between U and t[l]); the same bits as the per-step kernels.
  const TileLevel* tl = tile_at<T>(h, l);
  const bool tile_pre = zero_init && tile_presmooth<T>(h, l);
  // From u = 0 the first red half-sweep needs no stencil (k_first_half_zero); after it,
  // or after red_done, the black half-sweep writes every unknown of U.
  if (zero_init && !red_done && !tile_pre) {
    if (h->opt.smoother == MG_SMOOTH_REDBLACK && !fused_sweeps<T>(h) && h->opt.nu1 >= 1) {
      Bracket b(h, l, MG_KERNEL_SMOOTH, c.s);
      LAUNCH(h, 1, launch_first_half_zero<T>(H.L[l], F, H.t[l], 1, c.s));
      red_done = true;
    } else {
      CK(cudaMemsetAsync(U, 0, level_bytes(storage_of<T>(h->host[l], l), sizeof(T)), c.s));
    }
  }
  // Tile-kernel sweeps flip between U and t[l]; an odd number of them is evened out by
  // an out-of-place interpolation so that the level ends in U.
  T* cur = U;
  T* oth = H.t[l];
  const bool flips = fused_sweeps<T>(h);
  if (tile_pre) {
    Bracket b(h, l, MG_KERNEL_SMOOTH, c.s);
    LAUNCH(h, 1, launch_tile_presmooth(*tl, f32(H.L[l]), c.exact, (float*)U, status_word(h), c.s));
  } else {
    int k0 = 0;
    if (red_done) {
      Bracket b(h, l, MG_KERNEL_SMOOTH, c.s);
      LAUNCH(h, 1, launch_half_sweep<T>(H.L[l], c.exact, H.t[l], F, cur, 0, c.s));
      k0 = 1;
    }
    for (int k = k0; k < h->opt.nu1; ++k)
      if ((st = cycle_sweep<T>(c, l, cur, oth, F)) != MG_OK) return st;
  }
  // The restriction also writes the coarse level's first (zero-start) half-sweep when
  // that level runs as separate launches (and does not start with a tile presmooth).
  const bool coarse_red = l + 1 != lmax && l + 1 != H.tail_level && h->opt.smoother == MG_SMOOTH_REDBLACK &&
                          !fused_sweeps<T>(h) && h->opt.nu1 >= 1 && !tile_presmooth<T>(h, l + 1);
  if (tl && cur == U && (h->transfer[l] == kRbAxisToRot || h->transfer[l] == kRbRotToAxis)) {
    Bracket b(h, l, MG_KERNEL_RESIDUAL, c.s);
    LAUNCH(h, 1, launch_tile_res_restrict(*tl, f32(H.L[l]), f32(H.L[l + 1]), c.exact,
                                          (float*)H.f[l + 1], coarse_red ? (float*)H.t[l + 1] : nullptr,
                                          status_word(h), c.s));
  } else {
    {
      Bracket b(h, l, MG_KERNEL_RESIDUAL, c.s);
      LAUNCH(h, 1, launch_residual<T>(H.L[l], c.exact, cur, F, H.d[l], c.s));
    }
    Bracket b(h, l, MG_KERNEL_RESTRICT, c.s);
    LAUNCH(h, 1, launch_restrict<T>(H.L[l], H.L[l + 1], h->transfer[l], c.exact, H.d[l], H.f[l + 1], c.s,
                                    coarse_red ? H.t[l + 1] : nullptr));
  }
  if (l + 1 == lmax) {
    if (H.dense.m > 0)
      LAUNCH(h, 1, launch_coarsest_dense<T>(H.dense, H.L[lmax], c.exact, H.f[lmax], H.d[lmax], H.u[lmax], c.s));
    else
      LAUNCH(h, 1, launch_coarsest<T>(H.coarsest_idx, H.coarsest_a, H.coarsest_zero, H.f[lmax], H.u[lmax], c.s));
  } else {
    for (int g = 0; g < gamma_at(h, l); ++g)
      if ((st = cycle_level<T>(c, l + 1, H.u[l + 1], H.f[l + 1], g == 0, coarse_red && g == 0)) != MG_OK) return st;
  }
  // tile post-smoothing: sweeps ping-pong U <-> t[l], so an odd count starts from an
  // out-of-place interpolation into t[l]
  const bool tile_post = tl && h->opt.smoother == MG_SMOOTH_REDBLACK && cur == U;
  {
    Bracket b(h, l, MG_KERNEL_PROLONG, c.s);
    if ((flips || tile_post) && ((tile_post ? h->opt.nu2 : h->opt.nu1 + h->opt.nu2) & 1)) {
      LAUNCH(h, 1, launch_prolong_add<T>(H.L[l], H.L[l + 1], h->transfer[l], c.exact, oth, H.u[l + 1], c.s, cur));
      std::swap(cur, oth);
    } else {
      LAUNCH(h, 1, launch_prolong_add<T>(H.L[l], H.L[l + 1], h->transfer[l], c.exact, cur, H.u[l + 1], c.s));
    }
  }
  for (int k = 0; k < h->opt.nu2; ++k) {
    if (tile_post) {
      Bracket b(h, l, MG_KERNEL_SMOOTH, c.s);
      LAUNCH(h, 1, launch_tile_sweep(*tl, f32(H.L[l]), c.exact, cur == H.t[l],
                                     (float*)oth, status_word(h), c.s));
      std::swap(cur, oth);
    } else if ((st = cycle_sweep<T>(c, l, cur, oth, F)) != MG_OK) {
      return st;
    }
  }
  return cur == U ? MG_OK : MG_ERR_INVALID;
}

mg_status read_scalar(mg_handle* h, cudaStream_t s, double* out) {
  CK(cudaMemcpyAsync(h->hscalar, h->scalar, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *out = *h->hscalar;
  if (*reinterpret_cast<const int*>(h->hscalar + 1) != 0) return MG_ERR_TIMEOUT;
  return MG_OK;
}

mg_status rel_residual(mg_handle* h, const Ctx& c, const double* U, const double* F, double fn2,
                       double* out) {
  {
    Bracket b(h, 0, MG_KERNEL_NORM, c.s);
    LAUNCH(h, 2, launch_resnorm<double>(h->h64.L[0], c.exact, U, F, h->partial, h->scalar, c.s));
  }
  double r2;
  mg_status st = read_scalar(h, c.s, &r2);
  if (st != MG_OK) return st;
  *out = std::sqrt(r2) / std::sqrt(fn2);
  if (!std::isfinite(*out)) return MG_ERR_NONFINITE;
  return MG_OK;
}

// Whether the FP64 solve lets each residual-norm kernel also do the first half-sweep of
// the next cycle (k_resnorm_red): red-black smoothing with half-sweep kernels, at least
// one pre-smoothing sweep, and a finest level outside the small-level tail.
bool norm_takes_red(const mg_handle* h) {
  return h->opt.smoother == MG_SMOOTH_REDBLACK && !fused_sweeps<double>(h) && h->opt.nu1 >= 1 &&
         h->h64.tail_level != 0;
}

// rel_residual, and t[0] = U with its red nodes relaxed (discarded if no cycle follows).
mg_status rel_residual_red(mg_handle* h, const Ctx& c, const double* U, const double* F, double fn2,
                           double* out) {
  {
    Bracket b(h, 0, MG_KERNEL_NORM, c.s);
    LAUNCH(h, 2, launch_resnorm_red<double>(h->h64.L[0], c.exact, U, F, h->h64.t[0], 1, h->partial, h->scalar,
                                            c.s));
  }
  double r2;
  mg_status st = read_scalar(h, c.s, &r2);
  if (st != MG_OK) return st;
  *out = std::sqrt(r2) / std::sqrt(fn2);
  if (!std::isfinite(*out)) return MG_ERR_NONFINITE;
  return MG_OK;
}

mg_status f_norm2(mg_handle* h, cudaStream_t s, const double* F, double* out) {
  LAUNCH(h, 2, launch_sumsq<double>(h->h64.L[0], F, h->partial, h->scalar, s));
  mg_status st = read_scalar(h, s, out);
  if (st != MG_OK) return st;
  if (!std::isfinite(*out)) return MG_ERR_NONFINITE;
  if (*out == 0.0) return MG_ERR_INVALID;
  return MG_OK;
}

// Level descriptors and buffers of one precision. With caller_level0 the finest
// level's u and f are the caller's arrays (FP64 path); otherwise all four arrays are
// allocated (FP32 inner hierarchy of the mixed-precision path).
template <typename T>
mg_status alloc_hier(mg_handle* h, bool caller_level0) {
  Hier<T>& H = hier<T>(h);
  const int nl = (int)h->host.size();
  H.L.resize(nl);
  H.u.assign(nl, nullptr);
  H.t.assign(nl, nullptr);
  H.f.assign(nl, nullptr);
  H.d.assign(nl, nullptr);
  mg_status st;
  for (int l = 0; l < nl; ++l) {
    const int bf16 = (!caller_level0 && l < h->opt.bf16_levels) ? 1 : 0;
    const HostLevel S = storage_of<T>(h->host[l], l);
    if ((st = upload_level<T>(h, S, H.L[l], bf16)) != MG_OK) return st;
    const size_t b = level_bytes(S, sizeof(T));
    if (l > 0 || !caller_level0) {
      if ((st = device_alloc(h, (void**)&H.u[l], b)) != MG_OK) return st;
      if ((st = device_alloc(h, (void**)&H.f[l], b)) != MG_OK) return st;
    }
    if ((st = device_alloc(h, (void**)&H.t[l], b)) != MG_OK) return st;
    if ((st = device_alloc(h, (void**)&H.d[l], b)) != MG_OK) return st;
  }
  return MG_OK;
}

// Tail program for cycle_level(l, zero_init = true): the same op sequence the
// per-level launches would make. Nested levels start from u = 0 with the stencil-free
// first half-sweep (kOpSmooth, z = 1); the top level keeps its zeroing op, which the
// launch skips to continue from u.
void emit_tail(const mg_handle* h, int l, bool zero, std::vector<int4>& prog, bool top = false) {
  const int lmax = (int)h->host.size() - 1;
  const bool zs = zero && !top && h->opt.smoother == MG_SMOOTH_REDBLACK && h->opt.nu1 >= 1;
  if (zero && !zs) prog.push_back(make_int4(kOpZero, l, 0, 0));
  for (int k = 0; k < h->opt.nu1; ++k) prog.push_back(make_int4(kOpSmooth, l, zs && k == 0 ? 1 : 0, 0));
  prog.push_back(make_int4(kOpResRestrict, l, 0, 0));
  if (l + 1 == lmax) {
    prog.push_back(make_int4(kOpCoarsest, lmax, 0, 0));
  } else {
    for (int g = 0; g < gamma_at(h, l); ++g) emit_tail(h, l + 1, g == 0, prog);
  }
  prog.push_back(make_int4(kOpProlong, l, 0, 0));
  for (int k = 0; k < h->opt.nu2; ++k) prog.push_back(make_int4(kOpSmooth, l, 0, 0));
}

// Hand every level from the first one (below the finest) with at most
// `max_unknowns` unknowns down to the coarsest to the tail kernel.
// smem_elems > 0: instead of the unknowns threshold, take the first level (below the
// finest) from which all levels' u, t, f, d fit in that many shared-memory elements,
// and run the tail from shared memory.
template <typename T>
mg_status build_tail(mg_handle* h, int64_t max_unknowns, int64_t smem_elems = 0) {
  Hier<T>& H = hier<T>(h);
  const int nl = (int)h->host.size();
  int lt = -1;
  if (smem_elems > 0) {
    int64_t acc = 0;
    for (int l = nl - 1; l >= 1; --l) {
      acc += 4 * (int64_t)h->host[l].rows * h->host[l].cols;
      if (acc > smem_elems) break;
      if (l + 1 < nl) lt = l;
    }
  } else {
    for (int l = 1; l + 1 < nl; ++l)
      if (h->host[l].unknowns <= max_unknowns) { lt = l; break; }
  }
  if (lt < 0 || nl > kTailMaxLevels) return MG_OK;
  TailDesc<T> td;
  std::memset(&td, 0, sizeof(td));
  if (smem_elems > 0) {
    int off = 0;
    for (int l = lt; l < nl; ++l) {
      const int e = h->host[l].rows * h->host[l].cols;
      td.sm_u[l] = off;
      td.sm_t[l] = off + e;
      td.sm_f[l] = off + 2 * e;
      td.sm_d[l] = off + 3 * e;
      off += 4 * e;
    }
    if (tail_smem_bytes<T>(off, nl - lt) > kTailSmemMaxBytes) return MG_OK;  // no tail
    td.sm_top = lt;
    td.sm_elems = off;
    H.tail_smem = off;
  }
  for (int l = 0; l < nl; ++l) {
    td.L[l] = H.L[l].d;
    td.u[l] = H.u[l];
    td.t[l] = H.t[l];
    td.f[l] = H.f[l];
    td.d[l] = H.d[l];
    td.transfer[l] = l + 1 < nl ? h->transfer[l] : 0;
  }
  td.smoother = h->opt.smoother;
  td.nlev = nl;
  td.coarsest_idx = H.coarsest_idx;
  td.coarsest_a = H.coarsest_a;
  td.coarsest_zero = H.coarsest_zero;
  td.dense = H.dense;
  std::vector<int4> prog;
  emit_tail(h, lt, true, prog, true);
  mg_status st;
  if ((st = device_alloc(h, (void**)&H.d_tail, sizeof(td))) != MG_OK) return st;
  if ((st = device_alloc(h, (void**)&H.d_prog, prog.size() * sizeof(int4))) != MG_OK) return st;
  CK(cudaMemcpyAsync(H.d_tail, &td, sizeof(td), cudaMemcpyHostToDevice, h->priv));
  CK(cudaMemcpyAsync(H.d_prog, prog.data(), prog.size() * sizeof(int4), cudaMemcpyHostToDevice, h->priv));
  H.nops = (int)prog.size();
  H.tail_level = lt;
  H.tail_ctas = tail_ctas<T>(h->opt.fma_contract == 0);
  if (h->opt.tail_ctas > 0) H.tail_ctas = std::min(H.tail_ctas, (int)h->opt.tail_ctas);
  return MG_OK;
}

// Largest level (unknowns) run by the tail cluster (16 SMs). With the cycle in a
// CUDA graph a small level's full-grid launch costs little, and the tail's per-phase
// latency on 16 SMs only wins for the last few levels (measured on GB300).
constexpr int64_t kTailUnknownsFp64 = 256;
// FP32 inner hierarchies by default keep their small levels in one block's shared
// memory (up to 6K elements = 24 KB for u, t, f and d of every tail level). Measured on
// GB300, mixed solves (order 4, N(0,1) right-hand side; budget 4K / 6K / 8K / 12K / 16K /
// 24K elements): 257^2 n_min 16 to 1e-8 1.75 / 1.75 / 1.78 / 1.78 / 1.95 / 1.94 ms;
// 257^2 n_min 2 2.27 / 2.15 / 2.16 / 2.20 / 2.20 / 2.39; 2049^2 n_min 16 4.97-5.03 at 4K-12K,
// 5.15-5.16 above; 4097^2 n_min 16 to 1e-10 11.38-11.43 at 4K-12K, 11.64-11.65 above.
// A larger tail runs more levels on one SM, and their boundary-class term records no
// longer fit the L1 left beside the shared memory; no tail at all is slower still
// (257^2 n_min 2: 2.71 ms).
constexpr int64_t kTailSmemElemsFp32 = 6 * 1024;
// FP64 hierarchies by default use a shared-memory tail too, of 3K elements (24 KB);
// measured on GB300 (FP64 solve, 4097^2 / 513^2 / 129^2): cluster tail 65.8 / 8.45 /
// 5.55 ms, 3K 65.0 / 7.64 / 4.77, 6K 65.4 / 8.10 / 5.25, 12K 66.6 / 9.42 / 6.33.
// tail_unknowns > 0 selects the cluster tail with that threshold.
constexpr int64_t kTailSmemElemsFp64 = 3 * 1024;

// Power of two near 1 / rms of a residual with squared norm r2 over m unknowns, so
// that the FP32 copy of the residual stays far from underflow and overflow.
double ir_scale_for(double r2, int64_t m) {
  const double rms = std::sqrt(r2 / (double)std::max<int64_t>(m, 1));
  if (!(rms > 0.0) || !std::isfinite(rms)) return 1.0;
  return std::ldexp(1.0, -std::ilogb(rms));
}

// One refinement step of the mixed-precision solve: FP64 residual r = f - L u
// (also returns ||r||^2), then -- unless `norm_only` -- `inner_cycles` FP32 cycles
// on L e = r * scale from e = 0, and the FP64 update u += e / scale.
// Whether the refinement residual kernel also does the first (red) half-sweep of the
// FP32 cycle from e = 0 (conditions as norm_takes_red, on the FP32 hierarchy).
bool ir_takes_red(const mg_handle* h) {
  return h->opt.smoother == MG_SMOOTH_REDBLACK && !fused_sweeps<float>(h) && h->opt.nu1 >= 1 &&
         h->opt.inner_cycles >= 1 && h->h32.tail_level != 0 && !tile_presmooth<float>(h, 0);
}

mg_status ir_residual(const Ctx& c, double* u, const double* f, double* r2) {
  mg_handle* h = c.h;
  const bool red = ir_takes_red(h);
  {
    Bracket b(h, 0, MG_KERNEL_NORM, c.s);
    LAUNCH(h, 2, launch_ir_residual(h->h64.L[0], c.exact, u, f, h->h32.L[0], h->h32.f[0], h->ir_scale, h->partial,
                                    h->scalar, c.s, h->opt.bf16_levels > 0 ? 1 : 0, red ? h->h32.t[0] : nullptr));
  }
  return read_scalar(h, c.s, r2);
}

mg_status ir_correct(const Ctx& c, double* u) {
  mg_handle* h = c.h;
  mg_status st;
  const bool red = ir_takes_red(h);
  st = run_graph(c, h->g_inner32, nullptr, nullptr, [&]() -> mg_status {
    mg_status s2;
    for (int k = 0; k < h->opt.inner_cycles; ++k)
      if ((s2 = cycle_level<float>(c, 0, h->h32.u[0], h->h32.f[0], k == 0, red && k == 0)) != MG_OK) return s2;
    return MG_OK;
  });
  if (st != MG_OK) return st;
  LAUNCH(h, 1, launch_ir_update(h->h64.L[0], h->h32.L[0], u, h->h32.u[0], 1.0 / h->ir_scale, c.s));
  return MG_OK;
}

}  // namespace

extern "C" {

void mg_default_options(mg_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->omega = 1.0;
  o->nu1 = 1;
  o->nu2 = 1;
  o->gamma = 1;
  o->smoother = MG_SMOOTH_REDBLACK;
  o->n_min = 2;
  o->max_levels = 0;
  o->precision = MG_PREC_FP64;
  o->fma_contract = 0;
  o->inner_cycles = 1;
  o->tail_unknowns = 0;
  o->tail_ctas = 0;
  o->sweep_kernel = 0;
  o->bf16_levels = 0;
  o->boundary = MG_BOUNDARY_DIRICHLET;
  o->transfer_order = 2;
}

const char* mg_status_string(mg_status s) {
  switch (s) {
    case MG_OK: return "ok";
    case MG_ERR_INVALID: return "invalid argument";
    case MG_ERR_UNSUPPORTED: return "unsupported configuration";
    case MG_ERR_OOM: return "device out of memory";
    case MG_ERR_BUDGET: return "memory budget exceeded";
    case MG_ERR_CUDA: return "CUDA runtime error";
    case MG_ERR_NONFINITE: return "non-finite residual";
    case MG_ERR_NOT_CONVERGED: return "not converged";
    case MG_ERR_TIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

size_t mg_workspace_bytes(const mg_grid* grid, int order, mg_coarsening coarsening,
                          mg_coarse_op coarse_op, const mg_options* opt) {
  mg_options o;
  if (opt) o = *opt; else mg_default_options(&o);
  if (validate(grid, order, coarsening, coarse_op, o) != MG_OK) return 0;
  const auto shapes = level_shapes(grid->n, coarsening, coarsest_n(o), o.max_levels);
  size_t bytes = 0;
  for (size_t l = 0; l < shapes.size(); ++l) {
    const size_t rows = shapes[l].n + 1;
    const size_t cols = storage_cols(shapes[l].kind, shapes[l].n);
    const size_t pitch = l == 0 ? cols : round_pitch((int)cols);
    const size_t arrays = l == 0 ? 2 : 4;
    bytes += arrays * rows * pitch * sizeof(double);
    if (o.precision == MG_PREC_MIXED_FP32) bytes += 4 * rows * round_pitch((int)cols) * sizeof(float);
  }
  // dense coarsest factor (two m x m copies per precision) when the coarsest level has
  // several unknowns
  const LevelShape& c = shapes.back();
  const size_t mc = o.boundary == MG_BOUNDARY_PERIODIC ? 1
                    : c.kind == kAxis ? (size_t)(c.n - 1) * (c.n - 1)
                                      : ((size_t)(c.n - 1) * (c.n - 1) + 1) / 2;
  if (mc > 1) {
    bytes += 2 * mc * mc * sizeof(double) + mc * sizeof(int2);
    if (o.precision == MG_PREC_MIXED_FP32) bytes += 2 * mc * mc * sizeof(float) + mc * sizeof(int2);
  }
  return bytes;
}

mg_status mg_setup(const mg_grid* grid, int order, mg_coarsening coarsening, mg_coarse_op coarse_op,
                   const mg_options* opt, mg_handle** out) {
  if (!out) return MG_ERR_INVALID;
  *out = nullptr;
  mg_options o;
  if (opt) o = *opt; else mg_default_options(&o);
  mg_status st = validate(grid, order, coarsening, coarse_op, o);
  if (st != MG_OK) return st;
  mg_handle* h = new (std::nothrow) mg_handle();
  if (!h) return MG_ERR_OOM;
  h->N = grid->n;
  h->length = grid->length > 0.0 ? grid->length : 1.0;
  h->order = order;
  h->coarsening = coarsening;
  h->coarse_op = coarse_op;
  h->opt = o;
  const auto shapes = level_shapes(h->N, coarsening, coarsest_n(o), o.max_levels);
  if (!build_operators(h, shapes)) {
    delete h;
    return MG_ERR_UNSUPPORTED;
  }
  const int nl = (int)shapes.size();
  for (int l = 0; l + 1 < nl; ++l)
    h->transfer.push_back(transfer_of(coarsening, l, shapes[l].kind, o.transfer_order));
  for (const auto& L : h->host)
    if (L.c.size() > (size_t)kMaxTerms) { delete h; return MG_ERR_UNSUPPORTED; }
  auto fail = [&](mg_status s) { free_all(h); delete h; return s; };
  // Set-up work runs on the handle's own non-blocking stream: no device-wide
  // synchronisation, so other threads may keep capturing or running their streams.
  if (cudaStreamCreateWithFlags(&h->priv, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming) != cudaSuccess)
    return fail(MG_ERR_CUDA);
  const HostLevel& C = h->host.back();
  // several coarsest unknowns (n_min > 2, or a truncated hierarchy): the dense solve
  std::vector<double> cG;
  std::vector<int2> cij;
  if (C.unknowns != 1 &&
      (C.per || C.unknowns > kDenseMaxUnknowns || !dense_factor(C, cG, cij) || (int64_t)cij.size() != C.unknowns))
    return fail(MG_ERR_UNSUPPORTED);
  // Dirichlet: node (1, 1) with a_pp from its folded row; periodic: node (0, 0), whose
  // row is zero (the zero-mean solution is 0)
  const int64_t cidx = C.per ? 0 : (int64_t)1 * C.pitch + (C.shape.kind == kRot ? 0 : 1);
  const double ca = C.per ? 1.0
                          : (C.exact ? fold_row_x(C.Wx, C.shape.n, 1, 1) : fold_row(C.W, C.shape.n, 1, 1)).at(Key(0, 0)) * C.s;
  if ((st = alloc_hier<double>(h, /*caller_level0=*/true)) != MG_OK) return fail(st);
  h->h64.coarsest_idx = cidx;
  h->h64.coarsest_a = ca;
  h->h64.coarsest_zero = C.per;
  if (!cij.empty() && (st = upload_dense<double>(h, cG, cij, h->h64.dense)) != MG_OK) return fail(st);
  auto tail_limit = [&](int64_t dflt) -> int64_t {
    return o.tail_unknowns < 0 ? 0 : (o.tail_unknowns > 0 ? (int64_t)o.tail_unknowns : dflt);
  };
  if (o.tail_unknowns == 0 && kTailSmemElemsFp64 > 0) st = build_tail<double>(h, 0, kTailSmemElemsFp64);
  else st = build_tail<double>(h, tail_limit(kTailUnknownsFp64));
  if (st != MG_OK) return fail(st);
  if (o.precision == MG_PREC_MIXED_FP32) {
    if ((st = alloc_hier<float>(h, false)) != MG_OK) return fail(st);
    h->h32.coarsest_idx = cidx;
    h->h32.coarsest_a = (float)ca;
    h->h32.coarsest_zero = C.per;
    if (!cij.empty() && (st = upload_dense<float>(h, cG, cij, h->h32.dense)) != MG_OK) return fail(st);
    if (o.tail_unknowns == 0) st = build_tail<float>(h, 0, kTailSmemElemsFp32);
    else st = build_tail<float>(h, tail_limit(0));
    if (st != MG_OK) return fail(st);
    // TMA tile kernels on the large eligible FP32 levels above the tail (sweep_kernel 0)
    h->h32.tiles.assign(nl, TileLevel());
    if (o.sweep_kernel == 0 && o.smoother == MG_SMOOTH_REDBLACK)
      for (int l = 0; l + 1 < nl && (h->h32.tail_level < 0 || l < h->h32.tail_level); ++l)
        tile_setup(h->h32.tiles[l], h->h32.L[l], h->h32.u[l], h->h32.t[l], h->h32.f[l], o.nu1);
  }
  h->nblocks0 = resnorm_blocks<double>(h->h64.L[0]);
  if ((st = device_alloc(h, (void**)&h->partial, h->nblocks0 * sizeof(double))) != MG_OK) return fail(st);
  if ((st = device_alloc(h, (void**)&h->scalar, 64)) != MG_OK) return fail(st);
  if (cudaMallocHost((void**)&h->hscalar, 64) != cudaSuccess) return fail(MG_ERR_CUDA);
  h->host_allocs.push_back(h->hscalar);
  if (cudaStreamSynchronize(h->priv) != cudaSuccess) return fail(MG_ERR_CUDA);
  *out = h;
  return MG_OK;
}

mg_status mg_destroy(mg_handle* h) {
  if (!h) return MG_OK;
  free_all(h);
  delete h;
  return MG_OK;
}

int mg_num_levels(const mg_handle* h) { return h ? (int)h->host.size() : -1; }

mg_status mg_get_level_info(const mg_handle* h, int level, mg_level_info* out) {
  if (!h || !out || level < 0 || level >= (int)h->host.size()) return MG_ERR_INVALID;
  const HostLevel& L = h->host[level];
  out->kind = L.shape.kind;
  out->n = L.shape.n;
  out->rows = L.rows;
  out->cols = L.cols;
  out->pitch = L.pitch;
  out->unknowns = (int32_t)L.unknowns;
  out->nterms = (int32_t)L.c.size();
  out->periodic = L.per;
  return MG_OK;
}

mg_status mg_cycle(mg_handle* h, double* u, const double* f, double* rel_res_out, void* stream) {
  if (!h || !u || !f) return MG_ERR_INVALID;
  StreamScope scope(h, stream);
  Ctx c{h, scope.s, h->opt.fma_contract == 0};
  if (h->opt.dirichlet_data)  // the ping-pong array's boundary holds the data g too
    LAUNCH(h, 1, launch_copy_boundary<double>(h->h64.L[0], u, h->h64.t[0], c.s));
  else if (!h->host[0].per)
    LAUNCH(h, 1, launch_zero_boundary<double>(h->h64.L[0], u, c.s));
  mg_status st;
  double fn2;
  if (h->opt.precision == MG_PREC_MIXED_FP32) {
    if ((st = f_norm2(h, c.s, f, &fn2)) != MG_OK) return st;
    if (h->ir_scale == 0.0) h->ir_scale = ir_scale_for(fn2, h->host[0].unknowns);
    double r2;
    if ((st = ir_residual(c, u, f, &r2)) != MG_OK) return st;
    if (!std::isfinite(r2)) return MG_ERR_NONFINITE;
    h->ir_scale = ir_scale_for(r2, h->host[0].unknowns);
    if ((st = ir_residual(c, u, f, &r2)) != MG_OK) return st;  // residual at the chosen scale
    if ((st = ir_correct(c, u)) != MG_OK) return st;
  } else {
    st = run_graph(c, h->g_cycle64, u, f, [&]() { return cycle_level<double>(c, 0, u, f, false); });
    if (st != MG_OK) return st;
  }
  ++h->cycles;
  if (rel_res_out) {
    if (h->opt.precision != MG_PREC_MIXED_FP32 && (st = f_norm2(h, c.s, f, &fn2)) != MG_OK) return st;
    return rel_residual(h, c, u, f, fn2, rel_res_out);
  }
  return MG_OK;
}

mg_status mg_solve(mg_handle* h, double* u, const double* f, double rtol, int max_cycles,
                   int* cycles_out, double* history_out, void* stream) {
  if (!h || !u || !f || max_cycles < 0 || !(rtol >= 0.0)) return MG_ERR_INVALID;
  StreamScope scope(h, stream);
  Ctx c{h, scope.s, h->opt.fma_contract == 0};
  if (h->opt.dirichlet_data)  // the ping-pong array's boundary holds the data g too
    LAUNCH(h, 1, launch_copy_boundary<double>(h->h64.L[0], u, h->h64.t[0], c.s));
  else if (!h->host[0].per)
    LAUNCH(h, 1, launch_zero_boundary<double>(h->h64.L[0], u, c.s));
  double fn2, rr;
  mg_status st = f_norm2(h, c.s, f, &fn2);
  if (st != MG_OK) return st;
  int k = 0;
  if (h->opt.precision == MG_PREC_MIXED_FP32) {
    // Iterative refinement: each FP64 residual also feeds the next FP32 correction.
    h->ir_scale = ir_scale_for(fn2, h->host[0].unknowns);
    double r2;
    for (;;) {
      // FP64 residual at the scale predicted from the previous norm (the FP32 copy
      // stays in range as long as the residual moves by far less than 2^60 per step)
      if ((st = ir_residual(c, u, f, &r2)) != MG_OK) return st;
      rr = std::sqrt(r2) / std::sqrt(fn2);
      if (!std::isfinite(rr)) return MG_ERR_NONFINITE;
      if (history_out) history_out[k] = rr;
      if (k >= max_cycles || rr < rtol) break;
      const double want = ir_scale_for(r2, h->host[0].unknowns);
      if (want > 0x1p60 * h->ir_scale || want < 0x1p-60 * h->ir_scale) {
        h->ir_scale = want;  // redo the FP32 copy at a safe scale
        if ((st = ir_residual(c, u, f, &r2)) != MG_OK) return st;
      }
      if ((st = ir_correct(c, u)) != MG_OK) return st;
      h->ir_scale = want;
      ++k;
      ++h->cycles;
    }
  } else {
    // Each norm kernel also relaxes the red nodes into t[0]; the cycle graph then starts
    // with the black half-sweep (same bits as a full first sweep).
    const bool fuse = norm_takes_red(h);
    auto norm = [&]() { return fuse ? rel_residual_red(h, c, u, f, fn2, &rr) : rel_residual(h, c, u, f, fn2, &rr); };
    if ((st = norm()) != MG_OK) return st;
    if (history_out) history_out[0] = rr;
    while (k < max_cycles && rr >= rtol) {
      st = run_graph(c, fuse ? h->g_cycle64r : h->g_cycle64, u, f,
                     [&]() { return cycle_level<double>(c, 0, u, f, false, fuse); });
      if (st != MG_OK) return st;
      ++k;
      ++h->cycles;
      if ((st = norm()) != MG_OK) return st;
      if (history_out) history_out[k] = rr;
    }
  }
  if (cycles_out) *cycles_out = k;
  return rr < rtol ? MG_OK : MG_ERR_NOT_CONVERGED;
}

mg_status mg_solve_host(mg_handle* h, double* u_host, const double* f_host, double rtol, int max_cycles,
                        int* cycles_out, double* history_out, void* stream) {
  if (!h || !u_host || !f_host) return MG_ERR_INVALID;
  const size_t bytes = (size_t)(h->N + 1) * (h->N + 1) * sizeof(double);
  if (!h->host_u) {  // first call: the handle's device copies of u and f
    mg_status st;
    if ((st = device_alloc(h, (void**)&h->host_u, bytes)) != MG_OK) return st;
    if ((st = device_alloc(h, (void**)&h->host_f, bytes)) != MG_OK) return st;
    if (cudaStreamSynchronize(h->priv) != cudaSuccess) return MG_ERR_CUDA;  // the zero fills
  }
  const cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(h->host_f, f_host, bytes, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(h->host_u, u_host, bytes, cudaMemcpyHostToDevice, s));
  const mg_status st = mg_solve(h, h->host_u, h->host_f, rtol, max_cycles, cycles_out, history_out, stream);
  if (st != MG_OK && st != MG_ERR_NOT_CONVERGED) return st;
  CK(cudaMemcpyAsync(u_host, h->host_u, bytes, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return st;
}

mg_status mg_level_apply(mg_handle* h, int level, const double* u, double* out, void* stream) {
  if (!h || !u || !out || level < 0 || level >= (int)h->host.size()) return MG_ERR_INVALID;
  CK(launch_apply<double>(h->h64.L[level], h->opt.fma_contract == 0, u, out, (cudaStream_t)stream));
  return MG_OK;
}

mg_status mg_level_residual(mg_handle* h, int level, const double* u, const double* f, double* d,
                            void* stream) {
  if (!h || !u || !f || !d || level < 0 || level >= (int)h->host.size()) return MG_ERR_INVALID;
  CK(launch_residual<double>(h->h64.L[level], h->opt.fma_contract == 0, u, f, d, (cudaStream_t)stream));
  return MG_OK;
}

mg_status mg_level_smooth(mg_handle* h, int level, double* u, const double* f, int sweeps, void* stream) {
  if (!h || !u || !f || sweeps < 0 || level < 0 || level >= (int)h->host.size()) return MG_ERR_INVALID;
  Ctx c{h, (cudaStream_t)stream, h->opt.fma_contract == 0};
  for (int k = 0; k < sweeps; ++k) {
    mg_status st = smooth<double>(c, level, u, f);
    if (st != MG_OK) return st;
  }
  return MG_OK;
}

mg_status mg_level_restrict(mg_handle* h, int level, const double* d_fine, double* f_coarse, void* stream) {
  if (!h || !d_fine || !f_coarse || level < 0 || level + 1 >= (int)h->host.size()) return MG_ERR_INVALID;
  CK(launch_restrict<double>(h->h64.L[level], h->h64.L[level + 1], h->transfer[level], h->opt.fma_contract == 0,
                             d_fine, f_coarse, (cudaStream_t)stream));
  return MG_OK;
}

mg_status mg_level_prolong_add(mg_handle* h, int level, double* u_fine, const double* v_coarse, void* stream) {
  if (!h || !u_fine || !v_coarse || level < 0 || level + 1 >= (int)h->host.size()) return MG_ERR_INVALID;
  CK(launch_prolong_add<double>(h->h64.L[level], h->h64.L[level + 1], h->transfer[level], h->opt.fma_contract == 0,
                                u_fine, v_coarse, (cudaStream_t)stream));
  return MG_OK;
}

mg_status mg_get_counters(const mg_handle* h, mg_counters* out) {
  if (!h || !out) return MG_ERR_INVALID;
  out->launches = h->launches;
  out->cycles = h->cycles;
  return MG_OK;
}

mg_status mg_reset_counters(mg_handle* h) {
  if (!h) return MG_ERR_INVALID;
  h->launches = 0;
  h->cycles = 0;
  return MG_OK;
}

mg_status mg_set_timing(mg_handle* h, int enable) {
  if (!h || enable < 0 || enable > 2) return MG_ERR_INVALID;
  h->timing = enable;
  for (auto& u : h->ev_used) u = 0;
  return MG_OK;
}

mg_status mg_get_timing(mg_handle* h, int kernel_class, double* total_ms, int64_t* launches) {
  if (!h || kernel_class < 0 || kernel_class >= MG_KERNEL_CLASSES * (kTailMaxLevels + 1)) return MG_ERR_INVALID;
  double tot = 0.0;
  const size_t n = h->ev_used[kernel_class];
  for (size_t k = 0; k < n; ++k) {
    auto& e = h->ev[kernel_class][k];
    CK(cudaEventSynchronize(e.second));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e.first, e.second));
    tot += ms;
  }
  h->ev_used[kernel_class] = 0;
  if (total_ms) *total_ms = tot;
  if (launches) *launches = (int64_t)n;
  return MG_OK;
}

}  // extern "C"

namespace nsmg {
// Finest-level FP64 description of a handle (used by mg_rel_residual_static).
const LevelPair<double>* finest_level_fp64(const mg_handle* h, bool* exact) {
  if (!h || h->h64.L.empty()) return nullptr;
  if (exact) *exact = h->opt.fma_contract == 0;
  return &h->h64.L[0];
}
}  // namespace nsmg

// ===================================================================================
// Batched solves: many independent problems (each an mg_handle) advanced by a
// level-synchronous schedule. Every step of the V-cycle is one kernel launch covering
// that level of all problems that have it; problems converge independently (device
// active flags), so the whole inner cycle is captured once as a CUDA graph.
// ===================================================================================
namespace {

template <typename T>
struct BatchList {
  BatchLevel<T>* d_entries = nullptr;   // problems with level l + 1 (level l not the coarsest)
  int* d_prefix = nullptr;              // tiles over level l
  int* d_cprefix = nullptr;             // tiles over level l + 1 (restriction)
  int ne = 0, tiles = 0, ctiles = 0, rpt = 1;
  BatchLevel<T>* d_coarsest = nullptr;  // problems whose level l + 1 is the coarsest (one unknown)
  int nc = 0;
  BatchLevel<T>* d_coarsest_dense = nullptr;  // ... with several unknowns (dense solve)
  int ncd = 0;
  std::vector<BatchLevel<T>> host;
};

}  // namespace

struct mg_batch {
  std::vector<mg_handle*> hs;
  int count = 0, nl = 0;  // problems, most levels of any problem
  bool mixed = false, exact = true;
  int nu1 = 1, nu2 = 1, inner = 2;
  std::vector<BatchList<double>> lv64;
  std::vector<BatchList<float>> lv32;
  std::vector<BatchLevel<double>> fin;  // finest FP64 levels (norms, refinement)
  BatchLevel<double>* d_fin = nullptr;
  int* d_fin_prefix = nullptr;
  int fin_tiles = 0;
  std::vector<BatchLevel<double>> lv64_0;  // level-0 FP64 entries (u, f set per solve)
  int* d_active = nullptr;
  int* h_active = nullptr;
  double* d_scale = nullptr;
  double* h_scale = nullptr;
  double* d_partial = nullptr;
  double* d_norm2 = nullptr;
  double* h_norm2 = nullptr;
  cudaStream_t priv = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraphExec_t graph = nullptr;  // mixed: inner cycles; FP64: one cycle
  int64_t graph_kernels = 0;
  int64_t launches = 0;
  std::vector<void*> allocs, host_allocs;
  std::vector<int> rpt_choice;  // autotuned rows per thread per level
  // Hybrid schedule: the problems in `solo` are solved alone by mg_solve on the worker
  // streams `ws` (one host thread each); the others form the level-synchronous batch
  // `sync` (nullptr when every problem is solo). Empty `solo`: this batch is itself the
  // level-synchronous schedule over all problems.
  mg_batch* sync = nullptr;
  std::vector<int> solo, rest;  // problem indices; solo largest first
  std::vector<cudaStream_t> ws;
  std::vector<cudaEvent_t> wev;
};

namespace {

void batch_free(mg_batch* b) {
  if (b->sync) {
    cudaStreamSynchronize(b->sync->priv);
    batch_free(b->sync);
    delete b->sync;
    b->sync = nullptr;
  }
  for (cudaStream_t w : b->ws) {
    cudaStreamSynchronize(w);
    cudaStreamDestroy(w);
  }
  for (cudaEvent_t e : b->wev) cudaEventDestroy(e);
  b->ws.clear();
  b->wev.clear();
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->priv) cudaStreamDestroy(b->priv);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  for (void* p : b->allocs) cudaFree(p);
  for (void* p : b->host_allocs) cudaFreeHost(p);
  b->allocs.clear();
  b->host_allocs.clear();
}

mg_status batch_alloc(mg_batch* b, void** p, size_t bytes) {
  if (bytes == 0) bytes = 256;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA;
  }
  b->allocs.push_back(*p);
  return MG_OK;
}

template <typename T>
mg_status upload_vec(mg_batch* b, const std::vector<T>& v, T** d) {
  mg_status st = batch_alloc(b, (void**)d, std::max<size_t>(v.size(), 1) * sizeof(T));
  if (st != MG_OK) return st;
  if (!v.empty()) CK(cudaMemcpyAsync(*d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, b->priv));
  return MG_OK;
}

// Prefix sums of tiles for the entries of a list (level l or level l + 1 storage).
template <typename T>
std::vector<int> tile_prefix(const mg_batch* b, const std::vector<BatchLevel<T>>& es, int l, bool coarse, int rpt) {
  std::vector<int> p(1, 0);
  for (const auto& e : es) {
    const HostLevel& L = b->hs[e.problem]->host[coarse ? l + 1 : l];
    p.push_back(p.back() + batch_tiles(L.cols, L.rows, rpt));
  }
  return p;
}

// Level lists of one precision: entries for every level l that is not the coarsest
// of some problem, and the per-level coarsest lists.
template <typename T>
mg_status build_lists(mg_batch* b, std::vector<BatchList<T>>& lv) {
  lv.assign(b->nl, BatchList<T>());
  for (int l = 0; l + 1 < b->nl; ++l) {
    BatchList<T>& B = lv[l];
    std::vector<BatchLevel<T>> coarsest, coarsest_dense;
    for (int p = 0; p < b->count; ++p) {
      mg_handle* h = b->hs[p];
      Hier<T>& H = hier<T>(h);
      const int nlp = (int)h->host.size();
      if (l + 1 >= nlp) continue;
      BatchLevel<T> e;
      std::memset(&e, 0, sizeof(e));
      const HostLevel& L = h->host[l];
      e.L = H.L[l].d;
      e.Lc = H.L[l + 1].d;
      e.u = H.u[l];
      e.t = H.t[l];
      e.f = H.f[l];
      e.d = H.d[l];
      e.uc = H.u[l + 1];
      e.fc = H.f[l + 1];
      e.transfer = h->transfer[l];
      e.problem = p;
      e.cols = L.cols;
      e.rows = L.rows;
      e.n = L.shape.n;
      e.kind = L.shape.kind;
      e.tiles_x = (L.cols + kBatchCols - 1) / kBatchCols;
      e.ctiles_x = (h->host[l + 1].cols + kBatchCols - 1) / kBatchCols;
      e.coarsest_idx = H.coarsest_idx;
      e.coarsest_a = H.coarsest_a;
      e.dense = H.dense;
      e.dc = H.d[l + 1];
      B.host.push_back(e);
      if (l + 2 == nlp) (H.dense.m > 0 ? coarsest_dense : coarsest).push_back(e);
    }
    B.ne = (int)B.host.size();
    B.nc = (int)coarsest.size();
    B.ncd = (int)coarsest_dense.size();
    mg_status st;
    if ((st = upload_vec(b, B.host, &B.d_entries)) != MG_OK) return st;
    if ((st = upload_vec(b, coarsest, &B.d_coarsest)) != MG_OK) return st;
    if ((st = upload_vec(b, coarsest_dense, &B.d_coarsest_dense)) != MG_OK) return st;
  }
  return MG_OK;
}

template <typename T>
mg_status set_rpt(mg_batch* b, BatchList<T>& B, int l, int rpt) {
  const auto pf = tile_prefix(b, B.host, l, false, rpt);
  const auto pc = tile_prefix(b, B.host, l, true, rpt);
  mg_status st;
  if ((st = upload_vec(b, pf, &B.d_prefix)) != MG_OK) return st;
  if ((st = upload_vec(b, pc, &B.d_cprefix)) != MG_OK) return st;
  B.tiles = pf.back();
  B.ctiles = pc.back();
  B.rpt = rpt;
  return MG_OK;
}

// Autotuner: per level, rows per thread (1, 2 or 4) of the step kernels, chosen by
// timing the red half-sweep of the whole list with CUDA events.
template <typename T>
mg_status autotune(mg_batch* b, std::vector<BatchList<T>>& lv) {
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  b->rpt_choice.assign(b->nl, 1);
  for (int l = 0; l + 1 < b->nl; ++l) {
    BatchList<T>& B = lv[l];
    if (B.ne == 0) continue;
    int best = 1;
    float best_ms = 1e30f;
    for (int rpt : {1, 2, 4}) {
      mg_status st = set_rpt(b, B, l, rpt);
      if (st != MG_OK) return st;
      for (int rep = 0; rep < 4; ++rep) {
        if (rep == 1) CK(cudaEventRecord(e0, b->priv));
        CK(launch_batch_step<T>(kBHalfRed, B.d_entries, B.d_prefix, B.ne, B.tiles, rpt, b->d_active, b->exact,
                                b->priv));
      }
      CK(cudaEventRecord(e1, b->priv));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best_ms) {
        best_ms = ms;
        best = rpt;
      }
    }
    mg_status st = set_rpt(b, B, l, best);
    if (st != MG_OK) return st;
    b->rpt_choice[l] = best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return MG_OK;
}

#define BLAUNCH(b, expr)                            \
  do {                                              \
    ++(b)->launches;                                \
    if ((expr) != cudaSuccess) return MG_ERR_CUDA; \
  } while (0)

// One V-cycle of every active problem (level-synchronous), zero initial guess on the
// finest level when `zero0`.
template <typename T>
mg_status batch_cycle(mg_batch* b, std::vector<BatchList<T>>& lv, bool zero0, cudaStream_t s) {
  const int* act = b->d_active;
  for (int l = 0; l + 1 < b->nl; ++l) {
    BatchList<T>& B = lv[l];
    if (B.ne == 0) continue;
    // from u = 0 the first red half-sweep needs no stencil and replaces zeroing u
    const bool from_zero = l > 0 || zero0;
    if (from_zero && b->nu1 == 0)
      BLAUNCH(b, launch_batch_step<T>(kBZero, B.d_entries, B.d_prefix, B.ne, B.tiles, B.rpt, act, b->exact, s));
    for (int k = 0; k < b->nu1; ++k) {
      const int red_op = from_zero && k == 0 ? kBHalfRedZero : kBHalfRed;
      BLAUNCH(b, launch_batch_step<T>(red_op, B.d_entries, B.d_prefix, B.ne, B.tiles, B.rpt, act, b->exact, s));
      BLAUNCH(b, launch_batch_step<T>(kBHalfBlack, B.d_entries, B.d_prefix, B.ne, B.tiles, B.rpt, act, b->exact, s));
    }
    BLAUNCH(b, launch_batch_step<T>(kBResidual, B.d_entries, B.d_prefix, B.ne, B.tiles, B.rpt, act, b->exact, s));
    BLAUNCH(b, launch_batch_step<T>(kBRestrict, B.d_entries, B.d_cprefix, B.ne, B.ctiles, B.rpt, act, b->exact, s));
    if (B.nc > 0) BLAUNCH(b, launch_batch_step<T>(kBCoarsest, B.d_coarsest, nullptr, B.nc, 0, 1, act, b->exact, s));
    if (B.ncd > 0)
      BLAUNCH(b, launch_batch_step<T>(kBCoarsestDense, B.d_coarsest_dense, nullptr, B.ncd, 0, 1, act, b->exact, s));
  }
  for (int l = b->nl - 2; l >= 0; --l) {
    BatchList<T>& B = lv[l];
    if (B.ne == 0) continue;
    BLAUNCH(b, launch_batch_step<T>(kBProlong, B.d_entries, B.d_prefix, B.ne, B.tiles, B.rpt, act, b->exact, s));
    for (int k = 0; k < b->nu2; ++k) {
      BLAUNCH(b, launch_batch_step<T>(kBHalfRed, B.d_entries, B.d_prefix, B.ne, B.tiles, B.rpt, act, b->exact, s));
      BLAUNCH(b, launch_batch_step<T>(kBHalfBlack, B.d_entries, B.d_prefix, B.ne, B.tiles, B.rpt, act, b->exact, s));
    }
  }
  return MG_OK;
}

// The inner cycles (mixed) or one cycle (FP64) as a CUDA graph on b->priv.
mg_status batch_graph(mg_batch* b) {
  if (b->graph) return MG_OK;
  const int64_t before = b->launches;
  CK(cudaStreamBeginCapture(b->priv, cudaStreamCaptureModeThreadLocal));
  mg_status st = MG_OK;
  if (b->mixed) {
    for (int k = 0; k < b->inner && st == MG_OK; ++k) st = batch_cycle<float>(b, b->lv32, k == 0, b->priv);
  } else {
    st = batch_cycle<double>(b, b->lv64, false, b->priv);
  }
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->priv, &g);
  if (st != MG_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return st != MG_OK ? st : MG_ERR_CUDA;
  }
  const cudaError_t ei = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) return MG_ERR_CUDA;
  b->graph_kernels = b->launches - before;
  b->launches = before;
  return MG_OK;
}

// Level-synchronous schedule over every handle of the list (validated by the caller).
mg_status sync_create(mg_handle* const* handles, int count, mg_batch** out) {
  *out = nullptr;
  const mg_options& o0 = handles[0]->opt;
  mg_batch* b = new (std::nothrow) mg_batch();
  if (!b) return MG_ERR_OOM;
  auto fail = [&](mg_status s) { batch_free(b); delete b; return s; };
  b->hs.assign(handles, handles + count);
  b->count = count;
  b->mixed = o0.precision == MG_PREC_MIXED_FP32;
  b->exact = o0.fma_contract == 0;
  b->nu1 = o0.nu1;
  b->nu2 = o0.nu2;
  b->inner = o0.inner_cycles;
  for (auto* h : b->hs) b->nl = std::max(b->nl, (int)h->host.size());
  if (cudaStreamCreateWithFlags(&b->priv, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess)
    return fail(MG_ERR_CUDA);
  mg_status st;
  if ((st = batch_alloc(b, (void**)&b->d_active, count * sizeof(int))) != MG_OK) return fail(st);
  if ((st = batch_alloc(b, (void**)&b->d_scale, count * sizeof(double))) != MG_OK) return fail(st);
  if ((st = batch_alloc(b, (void**)&b->d_norm2, count * sizeof(double))) != MG_OK) return fail(st);
  if (cudaMallocHost((void**)&b->h_active, count * sizeof(int)) != cudaSuccess) return fail(MG_ERR_CUDA);
  b->host_allocs.push_back(b->h_active);
  if (cudaMallocHost((void**)&b->h_scale, count * sizeof(double)) != cudaSuccess) return fail(MG_ERR_CUDA);
  b->host_allocs.push_back(b->h_scale);
  if (cudaMallocHost((void**)&b->h_norm2, count * sizeof(double)) != cudaSuccess) return fail(MG_ERR_CUDA);
  b->host_allocs.push_back(b->h_norm2);
  for (int p = 0; p < count; ++p) b->h_active[p] = 1;
  if (cudaMemcpyAsync(b->d_active, b->h_active, count * sizeof(int), cudaMemcpyHostToDevice, b->priv) != cudaSuccess)
    return fail(MG_ERR_CUDA);
  // finest FP64 levels (norms, refinement); u / f filled in per solve
  for (int p = 0; p < count; ++p) {
    mg_handle* h = b->hs[p];
    BatchLevel<double> e;
    std::memset(&e, 0, sizeof(e));
    const HostLevel& L = h->host[0];
    e.L = h->h64.L[0].d;
    e.problem = p;
    e.cols = L.cols;
    e.rows = L.rows;
    e.n = L.shape.n;
    e.kind = L.shape.kind;
    e.tiles_x = (L.cols + kBatchCols - 1) / kBatchCols;
    if (b->mixed) {
      e.r32 = h->h32.f[0];
      e.e32 = h->h32.u[0];
      e.pitch32 = h->h32.L[0].h.pitch;
    }
    b->fin.push_back(e);
  }
  {
    std::vector<int> pf(1, 0);
    for (int p = 0; p < count; ++p) pf.push_back(pf.back() + batch_tiles(b->hs[p]->host[0].cols, b->hs[p]->host[0].rows, 1));
    b->fin_tiles = pf.back();
    if ((st = upload_vec(b, b->fin, &b->d_fin)) != MG_OK) return fail(st);
    if ((st = upload_vec(b, pf, &b->d_fin_prefix)) != MG_OK) return fail(st);
    if ((st = batch_alloc(b, (void**)&b->d_partial, std::max(b->fin_tiles, 1) * sizeof(double))) != MG_OK)
      return fail(st);
  }
  if (b->mixed) {
    if ((st = build_lists<float>(b, b->lv32)) != MG_OK) return fail(st);
    if ((st = autotune<float>(b, b->lv32)) != MG_OK) return fail(st);
  } else {
    if ((st = build_lists<double>(b, b->lv64)) != MG_OK) return fail(st);
    // level 0 runs on the caller's arrays; tune it on the handle's scratch arrays
    auto& B0 = b->lv64[0];
    b->lv64_0 = B0.host;
    for (auto& e : B0.host) {
      e.u = b->hs[e.problem]->h64.t[0];
      e.f = b->hs[e.problem]->h64.d[0];
    }
    if (cudaMemcpyAsync(B0.d_entries, B0.host.data(), B0.host.size() * sizeof(BatchLevel<double>),
                        cudaMemcpyHostToDevice, b->priv) != cudaSuccess)
      return fail(MG_ERR_CUDA);
    if ((st = autotune<double>(b, b->lv64)) != MG_OK) return fail(st);
    B0.host = b->lv64_0;
  }
  if (cudaStreamSynchronize(b->priv) != cudaSuccess) return fail(MG_ERR_CUDA);
  *out = b;
  return MG_OK;
}

mg_status sync_solve(mg_batch* b, double* const* u, const double* const* f, double rtol, int max_cycles,
                     int* cycles_out, double* rel_res_out, cudaStream_t user) {
  cudaStream_t s = b->priv;
  CK(cudaEventRecord(b->ev_in, user));
  CK(cudaStreamWaitEvent(s, b->ev_in, 0));
  struct Leave {
    mg_batch* b;
    cudaStream_t user;
    ~Leave() {
      cudaEventRecord(b->ev_out, b->priv);
      cudaStreamWaitEvent(user, b->ev_out, 0);
    }
  } leave{b, user};
  const int n = b->count;
  // caller arrays into the finest-level tables
  for (int p = 0; p < n; ++p) {
    b->fin[p].u = u[p];
    b->fin[p].f = const_cast<double*>(f[p]);
    ++b->launches;
    if (b->hs[p]->opt.dirichlet_data)  // the boundary of u holds the data g: into the ping-pong array
      CK(launch_copy_boundary<double>(b->hs[p]->h64.L[0], u[p], b->hs[p]->h64.t[0], s));
    else
      CK(launch_zero_boundary<double>(b->hs[p]->h64.L[0], u[p], s));
  }
  CK(cudaMemcpyAsync(b->d_fin, b->fin.data(), n * sizeof(BatchLevel<double>), cudaMemcpyHostToDevice, s));
  if (!b->mixed) {
    auto& B0 = b->lv64[0];
    for (auto& e : B0.host) {
      e.u = u[e.problem];
      e.f = const_cast<double*>(f[e.problem]);
    }
    CK(cudaMemcpyAsync(B0.d_entries, B0.host.data(), B0.host.size() * sizeof(BatchLevel<double>),
                       cudaMemcpyHostToDevice, s));
  }
  for (int p = 0; p < n; ++p) {
    b->h_active[p] = 1;
    b->h_scale[p] = 1.0;
  }
  CK(cudaMemcpyAsync(b->d_active, b->h_active, n * sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(b->d_scale, b->h_scale, n * sizeof(double), cudaMemcpyHostToDevice, s));
  // ||f||^2 per problem
  b->launches += 2;
  CK(launch_batch_norms(1, b->d_fin, b->d_fin_prefix, n, b->fin_tiles, b->d_active, b->d_scale, b->exact,
                        b->d_partial, b->d_norm2, s));
  CK(cudaMemcpyAsync(b->h_norm2, b->d_norm2, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  std::vector<double> fn2(b->h_norm2, b->h_norm2 + n), rr(n, 0.0);
  std::vector<int> cyc(n, 0);
  for (int p = 0; p < n; ++p) {
    if (!std::isfinite(fn2[p])) return MG_ERR_NONFINITE;
    if (fn2[p] == 0.0) return MG_ERR_INVALID;
    b->h_scale[p] = b->mixed ? ir_scale_for(fn2[p], b->hs[p]->host[0].unknowns) : 1.0;
  }
  mg_status st = batch_graph(b);
  if (st != MG_OK) return st;
  CK(cudaMemcpyAsync(b->d_scale, b->h_scale, n * sizeof(double), cudaMemcpyHostToDevice, s));
  int active = n;
  bool nonfinite = false;
  for (;;) {
    // residual norms (and, mixed, the scaled FP32 residual) of the active problems
    b->launches += 2;
    CK(launch_batch_norms(b->mixed ? 0 : 2, b->d_fin, b->d_fin_prefix, n, b->fin_tiles, b->d_active, b->d_scale,
                          b->exact, b->d_partial, b->d_norm2, s));
    CK(cudaMemcpyAsync(b->h_norm2, b->d_norm2, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::vector<double> next_scale(b->h_scale, b->h_scale + n);
    for (int p = 0; p < n; ++p) {
      if (!b->h_active[p]) continue;
      rr[p] = std::sqrt(b->h_norm2[p]) / std::sqrt(fn2[p]);
      if (!std::isfinite(rr[p])) nonfinite = true;
      if (!std::isfinite(rr[p]) || rr[p] < rtol || cyc[p] >= max_cycles) {
        b->h_active[p] = 0;
        --active;
      } else if (b->mixed) {
        next_scale[p] = ir_scale_for(b->h_norm2[p], b->hs[p]->host[0].unknowns);
      }
    }
    if (active == 0) break;
    CK(cudaMemcpyAsync(b->d_active, b->h_active, n * sizeof(int), cudaMemcpyHostToDevice, s));
    b->launches += b->graph_kernels;
    CK(cudaGraphLaunch(b->graph, s));
    if (b->mixed) {
      ++b->launches;
      CK(launch_batch_ir_update(b->d_fin, b->d_fin_prefix, n, b->fin_tiles, b->d_active, b->d_scale, s));
      std::copy(next_scale.begin(), next_scale.end(), b->h_scale);
      CK(cudaMemcpyAsync(b->d_scale, b->h_scale, n * sizeof(double), cudaMemcpyHostToDevice, s));
    }
    for (int p = 0; p < n; ++p)
      if (b->h_active[p]) ++cyc[p];
  }
  bool all = true;
  for (int p = 0; p < n; ++p) {
    if (cycles_out) cycles_out[p] = cyc[p];
    if (rel_res_out) rel_res_out[p] = rr[p];
    all = all && rr[p] < rtol;
  }
  if (nonfinite) return MG_ERR_NONFINITE;
  return all ? MG_OK : MG_ERR_NOT_CONVERGED;
}

// Problems at least this large (grid side N) are solved alone by default, on this many
// worker streams. Measured on 512 mixed-precision problems of sides 128..2048 (orders
// 2 and 4, n_min 16, rtol 1e-8) against 546 ms for the level-synchronous schedule
// alone: (1024, 4) 370 ms, (1024, 8) 310-313, (1024, 12) 306-310, (1024, 16) 305-308,
// (512, 12) 318-320, (2048, 12) 338-340.
constexpr int kSoloMinN = 1024;
constexpr int kSoloWorkers = 12;

int status_rank(mg_status s) { return s == MG_OK ? 0 : s == MG_ERR_NOT_CONVERGED ? 1 : 2; }

// Solo problems by mg_solve on the worker streams (each host thread takes the next
// unsolved problem, largest first) while the calling thread runs the level-synchronous
// part; the caller's stream waits for every stream at the end.
mg_status hybrid_solve(mg_batch* b, double* const* u, const double* const* f, double rtol, int max_cycles,
                       int* cycles_out, double* rel_res_out, cudaStream_t user) {
  const int ns = (int)b->solo.size(), nr = (int)b->rest.size(), nw = (int)b->ws.size();
  CK(cudaEventRecord(b->ev_in, user));
  for (cudaStream_t w : b->ws) CK(cudaStreamWaitEvent(w, b->ev_in, 0));
  std::vector<mg_status> st(ns, MG_OK);
  std::vector<int> cyc(ns, 0), rcyc(nr, 0);
  std::vector<double> rr(ns, NAN), rrr(nr, NAN);
  std::vector<int64_t> launched(nw, 0);
  std::atomic<int> next{0};
  auto work = [&](int t) {
    std::vector<double> hist;
    try {
      hist.resize(max_cycles + 1);
    } catch (...) {  // no memory for the history: this thread's problems report MG_ERR_OOM
      for (int i; (i = next.fetch_add(1)) < ns;) st[i] = MG_ERR_OOM;
      return;
    }
    for (int i; (i = next.fetch_add(1)) < ns;) {
      const int p = b->solo[i];
      mg_handle* h = b->hs[p];
      const int64_t l0 = h->launches;
      std::fill(hist.begin(), hist.end(), NAN);
      st[i] = mg_solve(h, u[p], f[p], rtol, max_cycles, &cyc[i], hist.data(), b->ws[t]);
      rr[i] = hist[cyc[i]];
      launched[t] += h->launches - l0;
    }
  };
  std::vector<std::thread> th;
  for (int t = 0; t < nw; ++t) {
    try {
      th.emplace_back(work, t);
    } catch (...) {  // no more threads: those started (or this one, below) take the rest
      break;
    }
  }
  mg_status sst = MG_OK;
  if (b->sync) {
    std::vector<double*> ur(nr);
    std::vector<const double*> fr(nr);
    for (int j = 0; j < nr; ++j) {
      ur[j] = u[b->rest[j]];
      fr[j] = f[b->rest[j]];
    }
    sst = sync_solve(b->sync, ur.data(), fr.data(), rtol, max_cycles, rcyc.data(), rrr.data(), user);
  }
  for (auto& x : th) x.join();
  if (th.empty()) work(0);
  for (int t = 0; t < nw; ++t) {
    b->launches += launched[t];
    CK(cudaEventRecord(b->wev[t], b->ws[t]));
    CK(cudaStreamWaitEvent(user, b->wev[t], 0));
  }
  for (int i = 0; i < ns; ++i) {
    if (cycles_out) cycles_out[b->solo[i]] = cyc[i];
    if (rel_res_out) rel_res_out[b->solo[i]] = rr[i];
  }
  for (int j = 0; j < nr; ++j) {
    if (cycles_out) cycles_out[b->rest[j]] = rcyc[j];
    if (rel_res_out) rel_res_out[b->rest[j]] = rrr[j];
  }
  // the first error (level-synchronous part, then solo problems by index), else
  // MG_ERR_NOT_CONVERGED if any problem missed rtol
  mg_status out = sst;
  std::vector<int> order(ns);
  for (int i = 0; i < ns; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int x, int y) { return b->solo[x] < b->solo[y]; });
  for (int i : order)
    if (status_rank(st[i]) > status_rank(out)) out = st[i];
  return out;
}

}  // namespace

extern "C" {

mg_status mg_batch_create_ex(mg_handle* const* handles, int count, const mg_batch_options* opt, mg_batch** out) {
  if (!handles || count <= 0 || !out) return MG_ERR_INVALID;
  *out = nullptr;
  const int solo_min_n = opt && opt->solo_min_n > 0 ? opt->solo_min_n : kSoloMinN;
  const int workers = opt && opt->workers > 0 ? opt->workers : kSoloWorkers;
  if ((opt && (opt->solo_min_n < 0 || opt->workers < 0)) || workers > 64) return MG_ERR_INVALID;
  if (!handles[0]) return MG_ERR_INVALID;
  const mg_options& o0 = handles[0]->opt;
  for (int p = 0; p < count; ++p) {
    const mg_handle* h = handles[p];
    if (!h) return MG_ERR_INVALID;
    const mg_options& o = h->opt;
    if (o.precision != o0.precision || o.nu1 != o0.nu1 || o.nu2 != o0.nu2 || o.fma_contract != o0.fma_contract ||
        (o.precision == MG_PREC_MIXED_FP32 && o.inner_cycles != o0.inner_cycles))
      return MG_ERR_INVALID;  // one schedule for the whole batch
    if (o.gamma != 1 || o.smoother != MG_SMOOTH_REDBLACK || o.bf16_levels != 0 ||
        o.boundary != MG_BOUNDARY_DIRICHLET || o.transfer_order != 2)
      return MG_ERR_UNSUPPORTED;
    if ((int)h->host.size() > kTailMaxLevels) return MG_ERR_UNSUPPORTED;
  }
  {  // each problem owns its handle's level arrays: a handle may appear once
    std::vector<const mg_handle*> seen(handles, handles + count);
    std::sort(seen.begin(), seen.end(), std::less<const mg_handle*>());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) return MG_ERR_INVALID;
  }
  std::vector<int> solo, rest;
  for (int p = 0; p < count; ++p) (handles[p]->N >= solo_min_n ? solo : rest).push_back(p);
  if (solo.empty()) return sync_create(handles, count, out);
  std::stable_sort(solo.begin(), solo.end(), [&](int x, int y) { return handles[x]->N > handles[y]->N; });
  mg_batch* b = new (std::nothrow) mg_batch();
  if (!b) return MG_ERR_OOM;
  auto fail = [&](mg_status s) { batch_free(b); delete b; return s; };
  b->hs.assign(handles, handles + count);
  b->count = count;
  b->solo = solo;
  b->rest = rest;
  if (cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess) return fail(MG_ERR_CUDA);
  for (int t = 0; t < std::min(workers, (int)solo.size()); ++t) {
    cudaStream_t w = nullptr;
    cudaEvent_t e = nullptr;
    if (cudaStreamCreateWithFlags(&w, cudaStreamNonBlocking) != cudaSuccess) return fail(MG_ERR_CUDA);
    b->ws.push_back(w);
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return fail(MG_ERR_CUDA);
    b->wev.push_back(e);
  }
  if (!rest.empty()) {
    std::vector<mg_handle*> hr;
    for (int p : rest) hr.push_back(handles[p]);
    mg_status st = sync_create(hr.data(), (int)hr.size(), &b->sync);
    if (st != MG_OK) return fail(st);
  }
  *out = b;
  return MG_OK;
}

mg_status mg_batch_create(mg_handle* const* handles, int count, mg_batch** out) {
  return mg_batch_create_ex(handles, count, nullptr, out);
}

mg_status mg_batch_destroy(mg_batch* b) {
  if (!b) return MG_OK;
  if (b->priv) cudaStreamSynchronize(b->priv);
  batch_free(b);
  delete b;
  return MG_OK;
}

mg_status mg_batch_solve(mg_batch* b, double* const* u, const double* const* f, double rtol, int max_cycles,
                         int* cycles_out, double* rel_res_out, void* stream) {
  if (!b || !u || !f || max_cycles < 0 || !(rtol >= 0.0)) return MG_ERR_INVALID;
  for (int p = 0; p < b->count; ++p)
    if (!u[p] || !f[p]) return MG_ERR_INVALID;
  if (!b->solo.empty()) return hybrid_solve(b, u, f, rtol, max_cycles, cycles_out, rel_res_out, (cudaStream_t)stream);
  return sync_solve(b, u, f, rtol, max_cycles, cycles_out, rel_res_out, (cudaStream_t)stream);
}

mg_status mg_batch_get_launches(const mg_batch* b, int64_t* launches) {
  if (!b || !launches) return MG_ERR_INVALID;
  *launches = b->launches + (b->sync ? b->sync->launches : 0);
  return MG_OK;
}

mg_status mg_solve_batched(mg_handle* const* handles, double* const* u, const double* const* f, int count,
                           double rtol, int max_cycles, int* cycles_out, double* rel_res_out, void* stream) {
  mg_batch* b = nullptr;
  mg_status st = mg_batch_create(handles, count, &b);
  if (st != MG_OK) return st;
  st = mg_batch_solve(b, u, f, rtol, max_cycles, cycles_out, rel_res_out, stream);
  mg_batch_destroy(b);
  return st;
}

}  // extern "C"
