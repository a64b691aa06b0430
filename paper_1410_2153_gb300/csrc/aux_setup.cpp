// Host part of the setup (first version): closure of the box tree
// (Sec. 3.2), the nested conforming auxiliary triangulations (Sec. 3.3) with
// the per-level data of the in-place V-cycle, the finest auxiliary
// coefficient and the Scott-Zhang transfer (Sec. 4.1).
//
// Boxes are named by depth and Morton prefix of their integer position; the
// closed tree is stored as one sorted array of split prefixes per depth.
// Auxiliary nodes are integer points of the 2^D lattice of the root box,
// named by their 64-bit Morton key; the free nodes of the finest level,
// sorted by key, are the auxiliary unknowns (every coarser level's nodes
// are among them because the grids are nested).
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <memory>
#include <thread>

#include "clip.h"
#include "internal.h"
#include "keyindex.h"

namespace asmg {

namespace {

inline uint64_t spread(uint64_t v) {
  v &= 0xffffffffULL;
  v = (v | (v << 16)) & 0x0000FFFF0000FFFFULL;
  v = (v | (v << 8)) & 0x00FF00FF00FF00FFULL;
  v = (v | (v << 4)) & 0x0F0F0F0F0F0F0F0FULL;
  v = (v | (v << 2)) & 0x3333333333333333ULL;
  v = (v | (v << 1)) & 0x5555555555555555ULL;
  return v;
}

inline uint64_t compact(uint64_t v) {
  v &= 0x5555555555555555ULL;
  v = (v | (v >> 1)) & 0x3333333333333333ULL;
  v = (v | (v >> 2)) & 0x0F0F0F0F0F0F0F0FULL;
  v = (v | (v >> 4)) & 0x00FF00FF00FF00FFULL;
  v = (v | (v >> 8)) & 0x0000FFFF0000FFFFULL;
  v = (v | (v >> 16)) & 0x00000000FFFFFFFFULL;
  return v;
}

inline uint64_t mort(uint64_t x, uint64_t y) { return spread(x) | (spread(y) << 1); }


struct BoxTree {
  int D = 31;
  std::vector<std::vector<uint64_t>> S;  // split prefixes per depth, sorted
  std::vector<KeyIndex> SI;              // lookup tables of S once it is final (index())

  void index() {
    SI.assign(S.size(), KeyIndex());
    for (size_t d = 0; d < S.size(); ++d) {
      int bits = 1;
      while (bits < 20 && ((size_t)1 << bits) < S[d].size()) ++bits;
      SI[d].build(S[d], bits);
    }
  }
  bool split(int d, uint64_t p) const {
    if (d < 0 || d >= (int)S.size()) return false;
    if (!SI.empty()) return SI[d].find(p) >= 0;
    return std::binary_search(S[d].begin(), S[d].end(), p);
  }
  bool exists(int d, uint64_t p) const { return d == 0 ? p == 0 : split(d - 1, p >> 2); }
  // edge neighbour at the same depth (dir 0 S, 1 E, 2 N, 3 W)
  bool nbr(int d, uint64_t p, int dir, uint64_t& q) const {
    static const int dx[4] = {0, 1, 0, -1}, dy[4] = {-1, 0, 1, 0};
    int64_t x = (int64_t)compact(p) + dx[dir], y = (int64_t)compact(p >> 1) + dy[dir];
    int64_t nb = 1LL << d;
    if (x < 0 || y < 0 || x >= nb || y >= nb) return false;
    q = mort((uint64_t)x, (uint64_t)y);
    return true;
  }
  // hanging midpoints of box (d, p) when it is shown at a level > d
  void hanging(int d, uint64_t p, bool h[4]) const {
    for (int e = 0; e < 4; ++e) {
      uint64_t q;
      h[e] = nbr(d, p, e, q) && split(d, q);
    }
  }
};

// Triangles of a box as lattice-key triples: SW-NE diagonal, or a fan about
// the centre through the hanging midpoints (Fig. "closure2").
void box_tris(const BoxTree& T, int d, uint64_t p, const bool h[4], std::vector<std::array<uint64_t, 3>>& out) {
  const uint64_t s = 1ULL << (T.D - d);
  const uint64_t x0 = compact(p) * s, y0 = compact(p >> 1) * s;
  const uint64_t SW = mort(x0, y0), SE = mort(x0 + s, y0), NE = mort(x0 + s, y0 + s), NW = mort(x0, y0 + s);
  if (!(h[0] || h[1] || h[2] || h[3])) {
    out.push_back({SW, SE, NE});
    out.push_back({SW, NE, NW});
    return;
  }
  const uint64_t m = s >> 1, C = mort(x0 + m, y0 + m);
  uint64_t ring[8];
  int n = 0;
  ring[n++] = SW;
  if (h[0]) ring[n++] = mort(x0 + m, y0);
  ring[n++] = SE;
  if (h[1]) ring[n++] = mort(x0 + s, y0 + m);
  ring[n++] = NE;
  if (h[2]) ring[n++] = mort(x0 + m, y0 + s);
  ring[n++] = NW;
  if (h[3]) ring[n++] = mort(x0, y0 + m);
  for (int i = 0; i < n; ++i) out.push_back({ring[i], ring[(i + 1) % n], C});
}

inline bool boundary_key(const BoxTree& T, uint64_t k) {
  uint64_t x = compact(k), y = compact(k >> 1), top = 1ULL << T.D;
  return x == 0 || y == 0 || x == top || y == top;
}



void sort_unique(std::vector<uint64_t>& v) {
  std::sort(v.begin(), v.end());
  v.erase(std::unique(v.begin(), v.end()), v.end());
}

// Boxes at depth d (children of the split boxes at d-1), ascending prefix.
std::vector<uint64_t> boxes_at(const BoxTree& T, int d) {
  if (d == 0) return {0};
  std::vector<uint64_t> b;
  if (d - 1 >= (int)T.S.size()) return b;
  b.reserve(T.S[d - 1].size() * 4);
  for (uint64_t p : T.S[d - 1])
    for (uint64_t c = 0; c < 4; ++c) b.push_back((p << 2) | c);
  return b;
}

using clip::clip_tri;
using clip::moments;
using clip::V2;

// Leaves of the closed tree meeting the closed lattice rectangle [lo, hi].
void leaves_in(const BoxTree& T, int64_t lox, int64_t loy, int64_t hix, int64_t hiy,
               std::vector<std::pair<int, uint64_t>>& out) {
  std::pair<int, uint64_t> st[256];
  int sp = 0;
  st[sp++] = {0, 0};
  while (sp) {
    auto b = st[--sp];
    int64_t s = 1LL << (T.D - b.first);
    int64_t x0 = (int64_t)compact(b.second) * s, y0 = (int64_t)compact(b.second >> 1) * s;
    if (x0 > hix || y0 > hiy || x0 + s < lox || y0 + s < loy) continue;
    if (!T.split(b.first, b.second)) {
      out.push_back(b);
      continue;
    }
    for (uint64_t c = 0; c < 4; ++c) st[sp++] = {b.first + 1, (b.second << 2) | c};
  }
}

constexpr unsigned MAX_THREADS = 64;

// A fine boundary segment of Gamma_D (mixed boundaries).
struct GSeg {
  double ax, ay, bx, by;
};

inline double orient2(double px, double py, double qx, double qy, double rx, double ry) {
  return (qx - px) * (ry - py) - (qy - py) * (rx - px);
}

// The closed segment s meets the interior of the CCW triangle K exactly when
// no line among K's edge lines and s's own line separates them, touching
// allowed (separating axes of the Minkowski difference of two convex
// polygons; only signs of orientations are used).
inline bool seg_cuts_open_tri(const double K[3][2], const GSeg& s) {
  for (int e = 0; e < 3; ++e) {
    const double* p = K[e];
    const double* q = K[(e + 1) % 3];
    if (orient2(p[0], p[1], q[0], q[1], s.ax, s.ay) <= 0 && orient2(p[0], p[1], q[0], q[1], s.bx, s.by) <= 0)
      return false;
  }
  int pos = 0, neg = 0;
  for (int v = 0; v < 3; ++v) {
    const double o = orient2(s.ax, s.ay, s.bx, s.by, K[v][0], K[v][1]);
    pos += o > 0;
    neg += o < 0;
  }
  return pos > 0 && neg > 0;
}

// The point (x, y) lies on the closed segment s.
inline bool on_seg(const GSeg& s, double x, double y) {
  return orient2(s.ax, s.ay, s.bx, s.by, x, y) == 0 && std::min(s.ax, s.bx) <= x && x <= std::max(s.ax, s.bx) &&
         std::min(s.ay, s.by) <= y && y <= std::max(s.ay, s.by);
}

// Gamma_D of a mixed problem: the fine boundary edges (edges of one element)
// with two Dirichlet endpoints, binned by bounding box on a uniform grid of
// gn x gn cells over the root box.
struct GammaD2 {
  std::vector<GSeg> seg;
  int gn = 1;
  double amin[2] = {0, 0}, L = 1;
  std::vector<int64_t> start = std::vector<int64_t>(2, 0);
  std::vector<int32_t> item;

  int cell(double v, int a, double slack) const {
    const double c = (v - amin[a]) / L * gn + slack;
    return (int)std::min<double>(gn - 1, std::max(0.0, std::floor(c)));
  }
  void build(const MeshHost& mesh, const TreeResult& tree) {
    amin[0] = tree.amin[0];
    amin[1] = tree.amin[1];
    L = tree.L;
    std::vector<std::array<int32_t, 2>> ed;
    ed.reserve(3 * mesh.ne);
    for (int64_t e = 0; e < mesh.ne; ++e)
      for (int k = 0; k < 3; ++k) {
        const int32_t a = mesh.E[3 * e + k], b = mesh.E[3 * e + (k + 1) % 3];
        ed.push_back({std::min(a, b), std::max(a, b)});
      }
    std::sort(ed.begin(), ed.end());
    for (size_t i = 0; i < ed.size();) {
      size_t j = i;
      while (j < ed.size() && ed[j] == ed[i]) ++j;
      const int32_t a = ed[i][0], b = ed[i][1];
      if (j - i == 1 && mesh.bflag[a] == 1 && mesh.bflag[b] == 1)
        seg.push_back(GSeg{mesh.X[2 * (int64_t)a], mesh.X[2 * (int64_t)a + 1], mesh.X[2 * (int64_t)b],
                           mesh.X[2 * (int64_t)b + 1]});
      i = j;
    }
    gn = std::max(1, std::min(1024, (int)std::sqrt((double)seg.size())));
    start.assign((size_t)gn * gn + 1, 0);
    for (int pass = 0; pass < 2; ++pass) {
      std::vector<int64_t> fill(start.begin(), start.end() - 1);
      for (size_t q = 0; q < seg.size(); ++q) {
        const GSeg& g = seg[q];
        const int x0 = cell(std::min(g.ax, g.bx), 0, -1e-9), x1 = cell(std::max(g.ax, g.bx), 0, 1e-9);
        const int y0 = cell(std::min(g.ay, g.by), 1, -1e-9), y1 = cell(std::max(g.ay, g.by), 1, 1e-9);
        for (int y = y0; y <= y1; ++y)
          for (int x = x0; x <= x1; ++x) {
            const int64_t ci = (int64_t)y * gn + x;
            if (pass == 0) start[ci + 1] += 1;
            else item[fill[ci]++] = (int32_t)q;
          }
      }
      if (pass == 0) {
        for (size_t ci = 0; ci + 1 < start.size(); ++ci) start[ci + 1] += start[ci];
        item.assign(start.back(), 0);
      }
    }
  }
  // f(segment) for the segments binned in the cells that the box [lo, hi]
  // meets; stops when f returns true
  template <class F>
  bool any(double lox, double loy, double hix, double hiy, F&& f) const {
    const int x0 = cell(lox, 0, -1e-9), x1 = cell(hix, 0, 1e-9);
    const int y0 = cell(loy, 1, -1e-9), y1 = cell(hiy, 1, 1e-9);
    for (int y = y0; y <= y1; ++y)
      for (int x = x0; x <= x1; ++x) {
        const int64_t ci = (int64_t)y * gn + x;
        for (int64_t q = start[ci]; q < start[ci + 1]; ++q)
          if (f(seg[item[q]])) return true;
      }
    return false;
  }
  // the interior of the CCW triangle K meets Gamma_D
  bool cuts(const double K[3][2]) const {
    if (seg.empty()) return false;
    const double lox = std::min({K[0][0], K[1][0], K[2][0]}), hix = std::max({K[0][0], K[1][0], K[2][0]});
    const double loy = std::min({K[0][1], K[1][1], K[2][1]}), hiy = std::max({K[0][1], K[1][1], K[2][1]});
    return any(lox, loy, hix, hiy, [&](const GSeg& g) { return seg_cuts_open_tri(K, g); });
  }
  // the point P lies on Gamma_D
  bool on(const double* P) const {
    if (seg.empty()) return false;
    return any(P[0], P[1], P[0], P[1], [&](const GSeg& g) { return on_seg(g, P[0], P[1]); });
  }
};

// f(thread, nthreads, begin, end) over contiguous ranges of [0, n), in order
template <class F>
void parallel_for(int64_t n, F f) {
  unsigned nt = std::max(1u, std::min(MAX_THREADS, std::thread::hardware_concurrency()));
  if (n < 4096) nt = 1;
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nt; ++t)
    th.emplace_back([&, t] { f(t, nt, n * t / nt, n * (t + 1) / nt); });
  for (auto& x : th) x.join();
}

// sorted unique union of per-thread lists (each part deduplicated in
// parallel first)
template <class V>
std::vector<V> merge_unique(std::vector<std::vector<V>>& parts) {
  auto su = [](std::vector<V>& v) {
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
  };
  std::vector<std::thread> th;
  for (auto& v : parts)
    if (!v.empty()) th.emplace_back([&v, &su] { su(v); });
  for (auto& x : th) x.join();
  // concatenate the sorted parts, merge them pairwise in parallel rounds,
  // then drop the duplicates that lay in different parts
  std::vector<V> all;
  std::vector<size_t> cut(1, 0);
  for (auto& v : parts) {
    if (v.empty()) continue;
    all.insert(all.end(), v.begin(), v.end());
    cut.push_back(all.size());
    std::vector<V>().swap(v);
  }
  const size_t np = cut.size() - 1;
  for (size_t w = 1; w < np; w *= 2) {
    std::vector<std::thread> mt;
    for (size_t t = 0; t + w < np; t += 2 * w) {
      const size_t a = cut[t], m = cut[t + w], b = cut[std::min(np, t + 2 * w)];
      mt.emplace_back([&all, a, m, b] { std::inplace_merge(all.begin() + a, all.begin() + m, all.begin() + b); });
    }
    for (auto& x : mt) x.join();
  }
  all.erase(std::unique(all.begin(), all.end()), all.end());
  return all;
}

}  // namespace

uint64_t lattice_key2(uint64_t x, uint64_t y) { return mort(x, y); }
void lattice_xy2(uint64_t key, uint64_t& x, uint64_t& y) {
  x = compact(key);
  y = compact(key >> 1);
}

void lattice_point(const TreeResult& t, uint64_t key, double* p) {
  p[0] = t.amin[0] + std::ldexp((double)compact(key), -t.D) * t.L;
  p[1] = t.amin[1] + std::ldexp((double)compact(key >> 1), -t.D) * t.L;
}

void build_aux_host(const MeshHost& mesh, const TreeResult& tree, const asmg_params& prm, AuxHost& out) {
  BoxTree T;
  T.D = tree.D;
  T.S = tree.split;

  // ---- Closure (Sec. 3.2, steps Mark/Close/Refine), finest level first:
  // a split box needs all four same-depth edge neighbours, so the parent of
  // every such neighbour is marked for refinement one level up.
  for (int d = (int)T.S.size() - 1; d >= 1; --d) {
    std::vector<uint64_t> add;
    for (uint64_t p : T.S[d])
      for (int e = 0; e < 4; ++e) {
        uint64_t q;
        if (T.nbr(d, p, e, q)) add.push_back(q >> 2);
      }
    std::vector<uint64_t>& up = T.S[d - 1];
    up.insert(up.end(), add.begin(), add.end());
    sort_unique(up);
  }
  out.split = T.S;
  const int J = (int)T.S.size();
  out.J = J;
  std::vector<std::vector<uint64_t>> BX(J + 1);  // boxes per depth, ascending prefix
  for (int d = 0; d <= J; ++d) BX[d] = boxes_at(T, d);
  // position of box p in BX[d] through a bucket index over the top key bits
  // (the same position as a binary search over the whole depth)
  std::vector<KeyIndex> BXI(J + 1);
  for (int d = 0; d <= J; ++d) {
    int bits = 1;
    while (bits < 20 && ((size_t)1 << bits) < BX[d].size()) ++bits;
    BXI[d].build(BX[d], bits);
  }
  auto box_at = [&](int d, uint64_t p) -> size_t {
    const int32_t i = BXI[d].find(p);
    return i >= 0 ? (size_t)i : (size_t)(std::lower_bound(BX[d].begin(), BX[d].end(), p) - BX[d].begin());
  };


  T.index();

  // ---- per level: changed boxes, new nodes and their parents, level sizes
  struct LevelInfo {
    std::vector<uint64_t> fanned;  // leaves at depth l-1 that gain hanging midpoints at level l
  };
  std::vector<LevelInfo> info(J + 1);
  out.nlevel.assign(J + 1, 0);
  std::vector<std::vector<std::array<uint64_t, 3>>> newnodes(J + 1);  // key, parent0, parent1
  std::vector<int64_t> nfree_new(J + 1, 0);
  std::atomic<int> next_nn(1);
  auto nn_worker = [&]() {
   for (;;) {
    const int l = next_nn.fetch_add(1);
    if (l > J) return;
    const int d = l - 1;
    const auto& bx = BX[d];
    std::vector<std::array<uint64_t, 3>> nn;
    auto add_box = [&](uint64_t p, bool split) {
      const uint64_t s = 1ULL << (T.D - d), m = s >> 1;
      const uint64_t x0 = compact(p) * s, y0 = compact(p >> 1) * s;
      const uint64_t SW = mort(x0, y0), SE = mort(x0 + s, y0), NE = mort(x0 + s, y0 + s), NW = mort(x0, y0 + s);
      nn.push_back({mort(x0 + m, y0 + m), SW, NE});  // centre: midpoint of the SW-NE diagonal
      if (split) {
        nn.push_back({mort(x0 + m, y0), SW, SE});
        nn.push_back({mort(x0 + s, y0 + m), SE, NE});
        nn.push_back({mort(x0 + m, y0 + s), NW, NE});
        nn.push_back({mort(x0, y0 + m), SW, NW});
      }
    };
    for (uint64_t p : bx) {
      bool sp = T.split(d, p);
      if (sp) {
        add_box(p, true);
      } else {
        bool h[4];
        T.hanging(d, p, h);
        if (h[0] || h[1] || h[2] || h[3]) {
          info[l].fanned.push_back(p);
          add_box(p, false);
        }
      }
    }
    std::sort(nn.begin(), nn.end());
    nn.erase(std::unique(nn.begin(), nn.end(), [](const std::array<uint64_t, 3>& a, const std::array<uint64_t, 3>& b) {
               return a[0] == b[0];
             }),
             nn.end());
    int64_t nfree = 0;
    for (auto& v : nn)
      if (!boundary_key(T, v[0])) ++nfree;
    nfree_new[l] = nfree;
    newnodes[l] = std::move(nn);
   }
  };
  {
    unsigned nt = std::max(1u, std::min(MAX_THREADS, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t) th.emplace_back(nn_worker);
    for (auto& x : th) x.join();
  }
  for (int l = 1; l <= J; ++l) out.nlevel[l] = out.nlevel[l - 1] + nfree_new[l];

  // ---- finest auxiliary coefficient: area-weighted mean of the fine
  // coefficients (exact clipping), accumulated per box half for coarser levels
  const bool varcoef = !mesh.coeff.empty();
  // R17: a domain that does not fill the root box uses the Dirichlet
  // auxiliary grids T^D_l (triangles inside Omega); the same clipping pass
  // then also measures how much of each triangle the fine elements cover
  const bool dgrid = !mesh.boxdomain && !mesh.mixed;
  // R18: a Neumann vertex selects the mixed grids T^M_l of the remark on
  // mixed boundary conditions (Sec. 3.4): the triangles whose interior meets
  // Omega and not Gamma_D, every node of them free except those on Gamma_D
  // or on a triangle cut by it.  They need the covered areas as well.
  const bool mixed = mesh.mixed;
  const bool cover = dgrid || mixed;
  // integral of a over the lower-right (0) / upper-left (1) diagonal halves
  // of every box, per depth, aligned with boxes_at(T, d); the covered area
  // of the same halves
  std::vector<std::vector<std::array<double, 2>>> half(J + 1), halfcov(J + 1);
  // integrals over the fan triangles of fanned leaves (key: sorted triangle)
  std::vector<std::pair<std::array<uint64_t, 3>, double>> fanint, fancov;
  auto tri_sorted = [](std::array<uint64_t, 3> t) {
    std::sort(t.begin(), t.end());
    return t;
  };
  // ---- the leaves' finest triangles (leaves numbered in depth-major box
  // order; first[d][i]: first triangle of box i of depth d, -1 if split), and
  // the node table of the device transfer build
  std::vector<std::vector<int64_t>> first(J + 1);
  std::vector<std::array<uint64_t, 3>> ftri;
  {
    SZTable& z = out.sz;
    z.dim = 2;
    z.D = T.D;
    z.amin[0] = tree.amin[0];
    z.amin[1] = tree.amin[1];
    z.L = tree.L;
    std::vector<int64_t> doff(J + 2, 0);
    for (int d = 0; d <= J; ++d) doff[d + 1] = doff[d] + (int64_t)BX[d].size();
    const int64_t nb = doff[J + 1];
    z.node_key.assign(nb, 0);
    z.node_pay.assign(nb, -1);
    std::vector<int32_t> ntri(nb, 0);
    for (int d = 0; d <= J; ++d) {
      const auto& bx = BX[d];
      parallel_for((int64_t)bx.size(), [&](unsigned, unsigned, int64_t b0, int64_t b1) {
        for (int64_t i = b0; i < b1; ++i) {
          const int64_t k = doff[d] + i;
          z.node_key[k] = bx[i];
          if (d < (int)T.S.size()) {
            auto it = std::lower_bound(T.S[d].begin(), T.S[d].end(), bx[i]);
            if (it != T.S[d].end() && *it == bx[i]) {
              z.node_pay[k] = doff[d + 1] + 4 * (int64_t)(it - T.S[d].begin());
              continue;
            }
          }
          bool h[4];
          T.hanging(d, bx[i], h);
          const int nh = (int)h[0] + (int)h[1] + (int)h[2] + (int)h[3];
          ntri[k] = nh ? 4 + nh : 2;
        }
      });
    }
    int64_t nleaf = 0, nt = 0;
    for (int d = 0; d <= J; ++d) {
      first[d].assign(BX[d].size(), -1);
      for (size_t i = 0; i < BX[d].size(); ++i) {
        const int64_t k = doff[d] + (int64_t)i;
        if (z.node_pay[k] >= 0) continue;
        z.node_pay[k] = -(nleaf + 1);
        z.leaf_first.push_back(nt);
        first[d][i] = nt;
        ++nleaf;
        nt += ntri[k];
      }
    }
    z.leaf_first.push_back(nt);
    ftri.resize(nt);
    for (int d = 0; d <= J; ++d) {
      const auto& bx = BX[d];
      parallel_for((int64_t)bx.size(), [&](unsigned, unsigned, int64_t b0, int64_t b1) {
        std::vector<std::array<uint64_t, 3>> kt;
        for (int64_t i = b0; i < b1; ++i) {
          if (first[d][i] < 0) continue;
          bool h[4];
          T.hanging(d, bx[i], h);
          kt.clear();
          box_tris(T, d, bx[i], h, kt);
          std::copy(kt.begin(), kt.end(), ftri.begin() + first[d][i]);
        }
      });
    }
  }
  if (varcoef || cover) {
    // clip every fine element against the finest triangles it meets
    std::vector<std::vector<std::pair<int64_t, double>>> contrib(64), ccontrib(64);
    parallel_for(mesh.ne, [&](unsigned t, unsigned, int64_t b, int64_t e) {
      auto& mine = contrib[t];
      std::vector<std::pair<int, uint64_t>> lv;
      std::vector<std::array<uint64_t, 3>> kt;
      const double sc = std::ldexp(1.0, T.D) / tree.L;
      for (int64_t el = b; el < e; ++el) {
        V2 P[3];
        double mnx = INFINITY, mny = INFINITY, mxx = -INFINITY, mxy = -INFINITY;
        for (int k = 0; k < 3; ++k) {
          int32_t v = mesh.E[3 * el + k];
          P[k] = V2{mesh.X[2 * v], mesh.X[2 * v + 1]};
          mnx = std::min(mnx, P[k].x); mxx = std::max(mxx, P[k].x);
          mny = std::min(mny, P[k].y); mxy = std::max(mxy, P[k].y);
        }
        lv.clear();
        leaves_in(T, (int64_t)std::floor((mnx - tree.amin[0]) * sc) - 2, (int64_t)std::floor((mny - tree.amin[1]) * sc) - 2,
                  (int64_t)std::ceil((mxx - tree.amin[0]) * sc) + 2, (int64_t)std::ceil((mxy - tree.amin[1]) * sc) + 2, lv);
        const V2 o = P[0];
        V2 Pl[3];
        for (int k = 0; k < 3; ++k) Pl[k] = V2{P[k].x - o.x, P[k].y - o.y};
        for (auto& lf : lv) {
          const size_t bi = box_at(lf.first, lf.second);
          const int64_t f0 = first[lf.first][bi];
          bool h[4];
          T.hanging(lf.first, lf.second, h);
          kt.clear();
          box_tris(T, lf.first, lf.second, h, kt);
          for (size_t q = 0; q < kt.size(); ++q) {
            V2 K[3];
            for (int k = 0; k < 3; ++k) {
              double p[2];
              lattice_point(tree, kt[q][k], p);
              K[k] = V2{p[0] - o.x, p[1] - o.y};
            }
            V2 poly[16];
            int m = clip_tri(Pl, 3, K, poly);
            if (m < 3) continue;
            double M[6];
            moments(poly, m, M);
            if (!(M[0] > 0)) continue;
            if (varcoef) mine.push_back({f0 + (int64_t)q, M[0] * mesh.coeff[el]});
            if (cover) ccontrib[t].push_back({f0 + (int64_t)q, M[0]});
          }
        }
      }
    });
    // reduce into finest-triangle integrals (fixed order: thread, then element)
    std::vector<double> I(ftri.size(), 0.0), C(ftri.size(), 0.0);
    for (auto& v : contrib)
      for (auto& pr : v) I[pr.first] += pr.second;
    for (auto& v : ccontrib)
      for (auto& pr : v) C[pr.first] += pr.second;
    // box-half integrals, bottom-up: a (half, fanint) and the covered area
    // (halfcov, fancov)
    for (int pass = 0; pass < 2; ++pass) {
    if (pass == 0 && !varcoef) continue;
    if (pass == 1 && !cover) continue;
    const std::vector<double>& IA = pass == 0 ? I : C;
    auto& H = pass == 0 ? half : halfcov;
    auto& FI = pass == 0 ? fanint : fancov;
    for (int d = J; d >= 0; --d) {
      const auto& bx = BX[d];
      H[d].assign(bx.size(), {0.0, 0.0});
      std::vector<std::vector<std::pair<std::array<uint64_t, 3>, double>>> fparts(MAX_THREADS);
      parallel_for((int64_t)bx.size(), [&](unsigned tix, unsigned, int64_t i0, int64_t i1) {
      for (int64_t i = i0; i < i1; ++i) {
        uint64_t p = bx[i];
        if (!T.split(d, p)) {
          bool h[4];
          T.hanging(d, p, h);
          std::vector<std::array<uint64_t, 3>> kt;
          box_tris(T, d, p, h, kt);
          const int64_t f0 = first[d][i];
          if (!(h[0] || h[1] || h[2] || h[3])) {
            H[d][i] = {IA[f0], IA[f0 + 1]};
          } else {
            // fan triangles on the S and E edges form the lower-right half
            const uint64_t s = 1ULL << (T.D - d);
            const uint64_t x0 = compact(p) * s, y0 = compact(p >> 1) * s;
            for (size_t k = 0; k < kt.size(); ++k) {
              uint64_t ax = compact(kt[k][0]), ay = compact(kt[k][0] >> 1);
              uint64_t bxx = compact(kt[k][1]), by = compact(kt[k][1] >> 1);
              bool lr = (ay == y0 && by == y0) || (ax == x0 + s && bxx == x0 + s);
              H[d][i][lr ? 0 : 1] += IA[f0 + k];
              fparts[tix].push_back({tri_sorted(kt[k]), IA[f0 + k]});
            }
          }
        } else {
          size_t j = box_at(d + 1, p << 2);
          // children: 0 SW, 1 SE, 2 NW, 3 NE (bit 0 = x, bit 1 = y)
          const auto& sw = H[d + 1][j];
          const auto& se = H[d + 1][j + 1];
          const auto& nw = H[d + 1][j + 2];
          const auto& ne = H[d + 1][j + 3];
          H[d][i][0] = sw[0] + se[0] + se[1] + ne[0];
          H[d][i][1] = sw[1] + nw[0] + nw[1] + ne[1];
        }
      }
      });
      for (auto& fp : fparts) FI.insert(FI.end(), fp.begin(), fp.end());
    }
    }
    std::sort(fanint.begin(), fanint.end());
    std::sort(fancov.begin(), fancov.end());
  }
  // covered area of one triangle of box (d, p) at a level where the box
  // shows as diagonal split (k = 0 lower-right, 1 upper-left) or as fan; the
  // triangle belongs to T^D_l when the fine elements cover (1 - 1e-9) of it
  auto tri_area = [&](const std::array<uint64_t, 3>& t) {
    double pa[2], pb[2], pc[2];
    lattice_point(tree, t[0], pa);
    lattice_point(tree, t[1], pb);
    lattice_point(tree, t[2], pc);
    return 0.5 * ((pb[0] - pa[0]) * (pc[1] - pa[1]) - (pc[0] - pa[0]) * (pb[1] - pa[1]));
  };
  // the value stored for one triangle in a box-half table H or a fan table FI
  auto tri_value = [&](const std::vector<std::vector<std::array<double, 2>>>& H,
                       const std::vector<std::pair<std::array<uint64_t, 3>, double>>& FI, int d, uint64_t p, bool diag,
                       int k, const std::array<uint64_t, 3>& t) -> double {
    if (diag) {
      const size_t i = box_at(d, p);
      return H[d][i][k];
    }
    auto it = std::lower_bound(FI.begin(), FI.end(), std::pair<std::array<uint64_t, 3>, double>(tri_sorted(t), -HUGE_VAL));
    return it->second;
  };
  // Gamma_D (mixed): the interior of lattice triangle t meets it; lattice
  // node x lies on it
  GammaD2 gdl;
  if (mixed) gdl.build(mesh, tree);
  auto gd_cuts = [&](const std::array<uint64_t, 3>& t) -> bool {
    double K[3][2];
    for (int v = 0; v < 3; ++v) lattice_point(tree, t[v], K[v]);
    return gdl.cuts(K);
  };
  auto on_gd = [&](uint64_t x) -> bool {
    double P[2];
    lattice_point(tree, x, P);
    return gdl.on(P);
  };
  // mixed: a triangle belongs to T^M_l when its interior meets Omega
  // (positive covered area) and not Gamma_D
  auto tri_kept = [&](int d, uint64_t p, bool diag, int k, const std::array<uint64_t, 3>& t) -> bool {
    return tri_value(halfcov, fancov, d, p, diag, k, t) > 1e-12 * tri_area(t) && !gd_cuts(t);
  };
  auto tri_inside = [&](int d, uint64_t p, bool diag, int k, const std::array<uint64_t, 3>& t) -> bool {
    if (mixed) return tri_kept(d, p, diag, k, t);
    if (!dgrid) return true;
    return tri_value(halfcov, fancov, d, p, diag, k, t) >= (1.0 - 1e-9) * tri_area(t);
  };
  // node x is free at level l (a vertex of sigma^(l) off the boundary of
  // Omega^D_l): every level-l triangle around it is inside.  The box shown
  // at level l around x in each quadrant holds those triangles.
  // Mixed: x is free when it is a node of a kept triangle, lies on no
  // triangle cut by Gamma_D and not on Gamma_D itself.
  auto free_at = [&](uint64_t x, int l, std::vector<std::array<uint64_t, 3>>& kt) -> bool {
    if (!mixed && boundary_key(T, x)) return false;
    const uint64_t X = compact(x), Y = compact(x >> 1);
    bool node = false;
    for (int q = 0; q < 4; ++q) {
      const bool px = q & 1, py = q & 2;
      int d = 0;
      uint64_t p = 0;
      while (d < l && T.split(d, p)) {
        const uint64_t sz = 1ULL << (T.D - d), hf = sz >> 1;
        const uint64_t x0 = compact(p) * sz, y0 = compact(p >> 1) * sz;
        const uint64_t cx = px ? (X >= x0 + hf) : (X > x0 + hf);
        const uint64_t cy = py ? (Y >= y0 + hf) : (Y > y0 + hf);
        p = (p << 2) | (cy << 1) | cx;
        ++d;
      }
      bool h[4] = {false, false, false, false};
      if (d < l) T.hanging(d, p, h);
      kt.clear();
      box_tris(T, d, p, h, kt);
      const bool diag = !(h[0] || h[1] || h[2] || h[3]);
      for (size_t k = 0; k < kt.size(); ++k) {
        if (kt[k][0] != x && kt[k][1] != x && kt[k][2] != x) continue;
        if (mixed) {
          if (gd_cuts(kt[k])) return false;
          if (tri_value(halfcov, fancov, d, p, diag, (int)k, kt[k]) > 1e-12 * tri_area(kt[k])) node = true;
          continue;
        }
        node = true;
        if (!tri_inside(d, p, diag, (int)k, kt[k])) return false;
      }
    }
    return node && !(mixed && on_gd(x));
  };

  // ---- finest-level nodes (aux unknowns): free at level J
  {
    std::vector<std::pair<int, uint64_t>> leaves;
    for (int d = 0; d <= J; ++d)
      for (uint64_t p : BX[d])
        if (!T.split(d, p)) leaves.push_back({d, p});
    // Every node of the closed (conforming, 2:1 balanced) grid lies in the
    // half-open square [x0, x0 + s) x [y0, y0 + s) of exactly one leaf, as its
    // SW corner, a hanging midpoint of its S or W edge, or the centre of its
    // fan; the nodes on the top and right sides of the root box belong to the
    // leaves along them.  Each leaf emits those nodes, so no key repeats.
    std::vector<std::vector<uint64_t>> part(MAX_THREADS);
    const uint64_t top = 1ULL << T.D;
    parallel_for((int64_t)leaves.size(), [&](unsigned t, unsigned, int64_t b0, int64_t b1) {
      auto put = [&](uint64_t x, uint64_t y) {
        const uint64_t k = mort(x, y);
        if (mixed || !boundary_key(T, k)) part[t].push_back(k);
      };
      for (int64_t q = b0; q < b1; ++q) {
        const int d = leaves[q].first;
        const uint64_t p = leaves[q].second;
        bool h[4];
        T.hanging(d, p, h);
        const uint64_t s = 1ULL << (T.D - d), m = s >> 1, x0 = compact(p) * s, y0 = compact(p >> 1) * s;
        put(x0, y0);
        if (h[0]) put(x0 + m, y0);
        if (h[3]) put(x0, y0 + m);
        if (h[0] || h[1] || h[2] || h[3]) put(x0 + m, y0 + m);
        if (y0 + s == top) {
          put(x0, top);
          if (h[2]) put(x0 + m, top);
        }
        if (x0 + s == top) {
          put(top, y0);
          if (h[1]) put(top, y0 + m);
        }
        if (x0 + s == top && y0 + s == top) put(top, top);
      }
    });
    out.aux_key = merge_unique(part);
  }
  if (dgrid) {
    // keep the vertices of inside level-J triangles that are free at J
    std::vector<int32_t> keep(out.aux_key.size(), 0);
    parallel_for((int64_t)out.aux_key.size(), [&](unsigned, unsigned, int64_t b0, int64_t b1) {
      std::vector<std::array<uint64_t, 3>> kt;
      for (int64_t q = b0; q < b1; ++q) keep[q] = free_at(out.aux_key[q], J, kt);
    });
    std::vector<uint64_t> ak;
    for (size_t q = 0; q < keep.size(); ++q)
      if (keep[q]) ak.push_back(out.aux_key[q]);
    out.aux_key.swap(ak);
  }
  const std::vector<uint64_t>& AK = out.aux_key;
  // first level at which each node is free: its birth level in a box domain;
  // with T^D_l the first level from its birth on whose triangles around it
  // are all inside (free at one level, free at all finer ones)
  std::vector<int32_t> phi, psi;
  if (mixed) {
    // every lattice node of sigma^(J) is a candidate: phi = first free level
    // from its birth on, psi = the first level after that where it is no
    // longer free (a node that leaves the grid does not come back)
    std::vector<std::pair<uint64_t, int32_t>> born;
    for (int l = 1; l <= J; ++l)
      for (auto& v : newnodes[l]) born.push_back({v[0], l});
    std::sort(born.begin(), born.end());
    const std::vector<uint64_t>& cand = out.aux_key;
    std::vector<int32_t> cphi(cand.size(), J + 1), cpsi(cand.size(), J + 1);
    parallel_for((int64_t)cand.size(), [&](unsigned, unsigned, int64_t b0, int64_t b1) {
      std::vector<std::array<uint64_t, 3>> kt;
      for (int64_t q = b0; q < b1; ++q) {
        auto it = std::lower_bound(born.begin(), born.end(), std::pair<uint64_t, int32_t>(cand[q], 0));
        int l = (it != born.end() && it->first == cand[q]) ? it->second : 0;
        while (l <= J && !free_at(cand[q], l, kt)) ++l;
        cphi[q] = l;
        if (l > J) continue;
        ++l;
        while (l <= J && free_at(cand[q], l, kt)) ++l;
        cpsi[q] = l;
      }
    });
    std::vector<uint64_t> ak;
    for (size_t q = 0; q < cand.size(); ++q)
      if (cphi[q] <= J) {
        ak.push_back(cand[q]);
        phi.push_back(cphi[q]);
        psi.push_back(cpsi[q]);
      }
    out.aux_key.swap(ak);
    out.nlevel.assign(J + 1, 0);
    for (int32_t f : phi) out.nlevel[f] += 1;
    for (int l = 1; l <= J; ++l) out.nlevel[l] += out.nlevel[l - 1];
    out.phi = phi;
    out.psi = psi;
  }
  if (dgrid) {
    std::vector<std::pair<uint64_t, int32_t>> born;
    for (int l = 1; l <= J; ++l)
      for (auto& v : newnodes[l]) born.push_back({v[0], l});
    std::sort(born.begin(), born.end());
    phi.assign(AK.size(), J + 1);
    parallel_for((int64_t)AK.size(), [&](unsigned, unsigned, int64_t b0, int64_t b1) {
      std::vector<std::array<uint64_t, 3>> kt;
      for (int64_t q = b0; q < b1; ++q) {
        auto it = std::lower_bound(born.begin(), born.end(), std::pair<uint64_t, int32_t>(AK[q], 0));
        int l = (it != born.end() && it->first == AK[q]) ? it->second : 0;
        while (l < J && !free_at(AK[q], l, kt)) ++l;
        phi[q] = l;
      }
    });
    out.nlevel.assign(J + 1, 0);
    for (int32_t f : phi) out.nlevel[f] += 1;
    for (int l = 1; l <= J; ++l) out.nlevel[l] += out.nlevel[l - 1];
  }
  KeyIndex AKI;
  AKI.build(AK, 20);
  // aux ID of node x at level l, or -1 where it is not a free node there
  auto level_id = [&](uint64_t x, int l) -> int32_t {
    if (mixed) {
      const int32_t id = AKI.find(x);
      return (id >= 0 && phi[id] <= l && l < psi[id]) ? id : -1;
    }
    if (boundary_key(T, x)) return -1;
    const int32_t id = AKI.find(x);
    if (dgrid && (id < 0 || phi[id] > l)) return -1;
    return id;
  };
  // coarsest level used: finest level with at most coarse_max_dofs free nodes
  out.c = 0;
  if (mixed) {
    // by the free nodes of each level (the nodes that left the grid excluded)
    std::vector<int64_t> nreal(J + 2, 0);
    for (size_t q = 0; q < phi.size(); ++q) {
      nreal[phi[q]] += 1;
      nreal[psi[q]] -= 1;
    }
    for (int l = 1; l <= J; ++l) nreal[l] += nreal[l - 1];
    for (int l = 0; l <= J; ++l)
      if (nreal[l] <= prm.coarse_max_dofs) out.c = l;
  } else {
    for (int l = 0; l <= J; ++l)
      if (out.nlevel[l] <= prm.coarse_max_dofs) out.c = l;
  }
  const int c = out.c;

  // coefficient of one triangle of box (d, p) at a level where the box shows
  // as diagonal split (k = 0 lower-right, 1 upper-left) or as fan
  // (the mean of a over the triangle, a = 0 outside Omega and a = 1 inside
  // when no coefficient is given)
  auto tri_coef = [&](int d, uint64_t p, bool diag, int k, const std::array<uint64_t, 3>& t) -> double {
    if (mixed) {
      // the mean of a over tau n Omega (R18)
      if (!varcoef) return 1.0;
      return tri_value(half, fanint, d, p, diag, k, t) / tri_value(halfcov, fancov, d, p, diag, k, t);
    }
    if (!varcoef && !dgrid) return 1.0;
    const auto& H = varcoef ? half : halfcov;
    const auto& FI = varcoef ? fanint : fancov;
    double pa[2], pb[2], pc[2];
    lattice_point(tree, t[0], pa);
    lattice_point(tree, t[1], pb);
    lattice_point(tree, t[2], pc);
    double area = 0.5 * ((pb[0] - pa[0]) * (pc[1] - pa[1]) - (pc[0] - pa[0]) * (pb[1] - pa[1]));
    double integral;
    if (diag) {
      size_t i = box_at(d, p);
      integral = H[d][i][k];
    } else {
      auto key = tri_sorted(t);
      auto it = std::lower_bound(FI.begin(), FI.end(), std::pair<std::array<uint64_t, 3>, double>(key, -HUGE_VAL));
      integral = it->second;
    }
    return integral / area;
  };

  // emit the triangles of box (d, p) as shown at level l
  auto emit_box = [&](int d, uint64_t p, int l, std::vector<int32_t>& ids, std::vector<uint64_t>& keys,
                      std::vector<double>& coef, std::vector<std::array<uint64_t, 3>>& kt) {
    bool h[4] = {false, false, false, false};
    if (d < l) T.hanging(d, p, h);
    kt.clear();
    box_tris(T, d, p, h, kt);
    bool diag = !(h[0] || h[1] || h[2] || h[3]);
    for (size_t k = 0; k < kt.size(); ++k) {
      if (!tri_inside(d, p, diag, (int)k, kt[k])) continue;  // outside Omega: not in T^D_l
      for (int v = 0; v < 3; ++v) {
        keys.push_back(kt[k][v]);
        ids.push_back(level_id(kt[k][v], l));
      }
      coef.push_back(tri_coef(d, p, diag, (int)k, kt[k]));
    }
  };

  // ---- coarsest level: all triangles of sigma^(c)
  {
    std::vector<std::array<uint64_t, 3>> ck;  // scratch
    for (int d = 0; d <= c; ++d) {
      for (uint64_t p : BX[d]) {
        if (d < c && T.split(d, p)) continue;
        emit_box(d, p, c, out.coarse_tri_id, out.coarse_tri_key, out.coarse_tri_coef, ck);
      }
    }
    for (auto id : out.coarse_tri_id)
      if (id >= 0) out.coarse_id.push_back(id);
    std::sort(out.coarse_id.begin(), out.coarse_id.end());
    out.coarse_id.erase(std::unique(out.coarse_id.begin(), out.coarse_id.end()), out.coarse_id.end());
  }

  // ---- levels c+1..J: smoothing sets, assembly triangles, new nodes; each
  // level in parallel over its changed boxes (per-thread lists merged,
  // sorted, unique), then over its relevant boxes (triangles concatenated in
  // order)
  out.levels.assign(std::max(0, J - c), AuxLevelHost());
  // local smoothing: the smoothing nodes (by aux ID) and the relevant boxes
  // (by index within their depth) of one level are marked in flag arrays and
  // gathered in ascending order, then the flags are cleared for the next level
  const bool local = prm.smoothing != 1 && !mixed;
  std::unique_ptr<std::atomic<uint8_t>[]> sflag;
  std::vector<std::unique_ptr<std::atomic<uint8_t>[]>> rflag(J + 1);
  if (local) {
    sflag.reset(new std::atomic<uint8_t>[AK.size() + 1]);
    for (size_t q = 0; q <= AK.size(); ++q) sflag[q].store(0, std::memory_order_relaxed);
    for (int dd = 0; dd <= J; ++dd) {
      rflag[dd].reset(new std::atomic<uint8_t>[BX[dd].size() + 1]);
      for (size_t q = 0; q <= BX[dd].size(); ++q) rflag[dd][q].store(0, std::memory_order_relaxed);
    }
  }
  for (int l = c + 1; l <= J; ++l) {
    AuxLevelHost& L = out.levels[l - (c + 1)];
    L.level = l;
    const int d = l - 1;
    const uint64_t s = 1ULL << (T.D - d);
    std::vector<uint64_t> changed = info[l].fanned;  // plus the split boxes
    changed.insert(changed.end(), T.S[d].begin(), T.S[d].end());
    sort_unique(changed);
    std::vector<uint64_t> sm;     // whole level: smoothing nodes by key
    std::vector<int32_t> smid;    // local: smoothing nodes by aux ID, ascending
    std::vector<std::pair<int, uint64_t>> rel;
    if (!local) {
      // every node of the level, every box shown at the level (always for
      // the mixed grids, which are not nested)
      for (int dd = 0; dd <= l; ++dd)
        for (uint64_t p : BX[dd])
          if (!(dd < l && T.split(dd, p))) rel.push_back({dd, p});
      std::vector<std::vector<uint64_t>> part(MAX_THREADS);
      parallel_for((int64_t)rel.size(), [&](unsigned t, unsigned, int64_t b0, int64_t b1) {
        std::vector<std::array<uint64_t, 3>> kt;
        for (int64_t q = b0; q < b1; ++q) {
          const int dd = rel[q].first;
          bool h[4] = {false, false, false, false};
          if (dd < l) T.hanging(dd, rel[q].second, h);
          kt.clear();
          box_tris(T, dd, rel[q].second, h, kt);
          for (auto& x : kt)
            for (int v = 0; v < 3; ++v)
              if (level_id(x[v], l) >= 0) part[t].push_back(x[v]);
        }
      });
      sm = merge_unique(part);
    } else {
      // N~_l: the corners and centres of the changed boxes, and the edge
      // midpoints of the split ones; relevant boxes: the changed boxes and the
      // level-l leaves around them
      auto mark_node = [&](int32_t id) {
        if (id >= 0) sflag[id].store(1, std::memory_order_relaxed);
      };
      auto mark_box = [&](int dd, uint64_t pp) {
        rflag[dd][box_at(dd, pp)].store(1, std::memory_order_relaxed);
      };
      parallel_for((int64_t)changed.size(), [&](unsigned, unsigned, int64_t b0, int64_t b1) {
        std::vector<std::array<uint64_t, 3>> kt;
        for (int64_t q = b0; q < b1; ++q) {
          const uint64_t p = changed[q];
          const uint64_t x0 = compact(p) * s, y0 = compact(p >> 1) * s, m = s >> 1;
          const bool sp = T.split(d, p);
          if (!dgrid) {
            for (int iy = 0; iy <= 2; ++iy)
              for (int ix = 0; ix <= 2; ++ix) {
                bool mid = (ix == 1) || (iy == 1);
                if (mid && !sp && !(ix == 1 && iy == 1)) continue;  // fanned leaf: corners and centre
                uint64_t k = mort(x0 + ix * m, y0 + iy * m);
                if (!boundary_key(T, k)) mark_node(AKI.find(k));
              }
          } else {
            // free vertices of the box's new triangles that lie inside Omega
            auto add_inside = [&](int dd, uint64_t pp, const bool* h) {
              kt.clear();
              box_tris(T, dd, pp, h, kt);
              const bool diag = !(h[0] || h[1] || h[2] || h[3]);
              for (size_t k = 0; k < kt.size(); ++k) {
                if (!tri_inside(dd, pp, diag, (int)k, kt[k])) continue;
                for (int v = 0; v < 3; ++v)
                  mark_node(level_id(kt[k][v], l));
              }
            };
            bool h[4] = {false, false, false, false};
            if (sp) {
              for (uint64_t ch = 0; ch < 4; ++ch) add_inside(d + 1, (p << 2) | ch, h);
            } else {
              T.hanging(d, p, h);
              add_inside(d, p, h);
            }
          }
          if (sp) {
            for (uint64_t ch = 0; ch < 4; ++ch) mark_box(d + 1, (p << 2) | ch);
          } else {
            mark_box(d, p);
          }
          const int64_t x = (int64_t)compact(p), y = (int64_t)compact(p >> 1), nb = 1LL << d;
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              if (!dx && !dy) continue;
              if (x + dx < 0 || y + dy < 0 || x + dx >= nb || y + dy >= nb) continue;
              int dd = d;
              uint64_t nq = mort((uint64_t)(x + dx), (uint64_t)(y + dy));
              while (!T.exists(dd, nq)) {
                --dd;
                nq >>= 2;
              }
              if (dd == d && T.split(d, nq)) {
                for (uint64_t ch = 0; ch < 4; ++ch) mark_box(d + 1, (nq << 2) | ch);
              } else {
                mark_box(dd, nq);
              }
            }
        }
      });
      // gather (contiguous ranges per thread, concatenated in order) and clear
      {
        std::vector<std::vector<int32_t>> sp(MAX_THREADS);
        parallel_for((int64_t)AK.size(), [&](unsigned t, unsigned, int64_t b0, int64_t b1) {
          for (int64_t q = b0; q < b1; ++q)
            if (sflag[q].load(std::memory_order_relaxed)) {
              sp[t].push_back((int32_t)q);
              sflag[q].store(0, std::memory_order_relaxed);
            }
        });
        for (auto& v : sp) smid.insert(smid.end(), v.begin(), v.end());
      }
      for (int dd = 0; dd <= d + 1; ++dd) {
        const auto& bx = BX[dd];
        std::vector<std::vector<std::pair<int, uint64_t>>> rp(MAX_THREADS);
        parallel_for((int64_t)bx.size(), [&](unsigned t, unsigned, int64_t b0, int64_t b1) {
          for (int64_t q = b0; q < b1; ++q)
            if (rflag[dd][q].load(std::memory_order_relaxed)) {
              rp[t].push_back({dd, bx[q]});
              rflag[dd][q].store(0, std::memory_order_relaxed);
            }
        });
        for (auto& v : rp) rel.insert(rel.end(), v.begin(), v.end());
      }
    }
    if (local) {
      L.smooth.swap(smid);
    } else {
      L.smooth.resize(sm.size());
      parallel_for((int64_t)sm.size(), [&](unsigned, unsigned, int64_t b0, int64_t b1) {
        for (int64_t q = b0; q < b1; ++q) L.smooth[q] = AKI.find(sm[q]);
      });
      std::sort(rel.begin(), rel.end());
      rel.erase(std::unique(rel.begin(), rel.end()), rel.end());
    }
    std::vector<std::vector<int32_t>> ids(MAX_THREADS);
    std::vector<std::vector<uint64_t>> keys(MAX_THREADS);
    std::vector<std::vector<double>> coefs(MAX_THREADS);
    parallel_for((int64_t)rel.size(), [&](unsigned t, unsigned, int64_t b0, int64_t b1) {
      std::vector<std::array<uint64_t, 3>> kt;  // scratch of this thread
      for (int64_t q = b0; q < b1; ++q) emit_box(rel[q].first, rel[q].second, l, ids[t], keys[t], coefs[t], kt);
    });
    // concatenate in thread order: sizes first, then one copy per part in parallel
    {
      std::vector<size_t> o3(MAX_THREADS + 1, 0), o1(MAX_THREADS + 1, 0);
      for (unsigned t = 0; t < MAX_THREADS; ++t) {
        o3[t + 1] = o3[t] + ids[t].size();
        o1[t + 1] = o1[t] + coefs[t].size();
      }
      L.tri_id.resize(o3[MAX_THREADS]);
      L.tri_key.resize(o3[MAX_THREADS]);
      L.tri_coef.resize(o1[MAX_THREADS]);
      std::vector<std::thread> th;
      for (unsigned t = 0; t < MAX_THREADS; ++t) {
        if (coefs[t].empty() && ids[t].empty()) continue;
        th.emplace_back([&, t] {
          std::copy(ids[t].begin(), ids[t].end(), L.tri_id.begin() + o3[t]);
          std::copy(keys[t].begin(), keys[t].end(), L.tri_key.begin() + o3[t]);
          std::copy(coefs[t].begin(), coefs[t].end(), L.tri_coef.begin() + o1[t]);
        });
      }
      for (auto& x : th) x.join();
    }
    if (mixed && mesh.nb_layers >= 0) {
      // Algorithm 3: J_{l,j} = the free nodes of the j-th layer of triangles
      // around Gamma_l
      for (uint64_t k : nb::near_boundary_nodes(3, L.tri_key, mesh.nb_layers)) {
        const int32_t id = level_id(k, l);
        if (id >= 0) L.nb_id.push_back(id);
      }
      std::sort(L.nb_id.begin(), L.nb_id.end());
      // A_l[J,J] from the level's kept simplices, factored for the exact
      // near-boundary solve
      std::vector<double> pts(L.tri_key.size() * 2);
      for (size_t k = 0; k < L.tri_key.size(); ++k) lattice_point(tree, L.tri_key[k], &pts[2 * k]);
      nb::assemble_block(2, L.tri_coef.size(), pts.data(), L.tri_coef.data(), L.tri_id.data(), L.nb_id, L.nb_ptr,
                         L.nb_col, L.nb_val);
      if (!nb::factor((int64_t)L.nb_id.size(), L.nb_ptr.data(), L.nb_col.data(), L.nb_val.data(), L.nb_fac))
        ASMG_FAIL(ASMG_ERR_BAD_MESH, "near-boundary block not positive definite");
    }
    // new nodes with their parents
    if (!dgrid && !mixed) {
      for (auto& v : newnodes[l]) {
        if (boundary_key(T, v[0])) continue;
        L.new_id.push_back(AKI.find(v[0]));
        L.new_p0.push_back(boundary_key(T, v[1]) ? -1 : AKI.find(v[1]));
        L.new_p1.push_back(boundary_key(T, v[2]) ? -1 : AKI.find(v[2]));
      }
    } else {
      // nodes free from level l on: born at l, the interpolant of the
      // level-(l-1) function at the edge midpoint (a parent off the free
      // nodes of l-1 contributes 0); born earlier on the boundary of
      // Omega^D_(l-1), where that function vanishes: no parents
      const auto& nn = newnodes[l];
      for (size_t q = 0; q < AK.size(); ++q) {
        if (phi[q] != l) continue;
        auto it = std::lower_bound(nn.begin(), nn.end(), std::array<uint64_t, 3>{AK[q], 0, 0});
        const bool born = it != nn.end() && (*it)[0] == AK[q];
        L.new_id.push_back((int32_t)q);
        L.new_p0.push_back(born ? level_id((*it)[1], l - 1) : -1);
        L.new_p1.push_back(born ? level_id((*it)[2], l - 1) : -1);
      }
    }
  }

  // ---- columns of the finest triangles for the device Scott-Zhang build
  // (Sec. 4.1): the aux ID of every vertex with a hat function at level J;
  // none on the triangles outside Omega^D_J
  {
    SZTable& z = out.sz;
    z.simp_key.resize(3 * ftri.size());
    z.simp_col.assign(3 * ftri.size(), -1);
    if (!ftri.empty()) std::memcpy(z.simp_key.data(), ftri.data(), ftri.size() * sizeof(ftri[0]));
    for (int d = 0; d <= J; ++d) {
      const auto& bx = BX[d];
      parallel_for((int64_t)bx.size(), [&](unsigned, unsigned, int64_t b0, int64_t b1) {
        for (int64_t i = b0; i < b1; ++i) {
          const int64_t f0 = first[d][i];
          if (f0 < 0) continue;
          bool h[4];
          T.hanging(d, bx[i], h);
          const int nh = (int)h[0] + (int)h[1] + (int)h[2] + (int)h[3];
          const int nt = nh ? 4 + nh : 2;
          for (int k = 0; k < nt; ++k) {
            const auto& t = ftri[f0 + k];
            if (!tri_inside(d, bx[i], nh == 0, k, t)) continue;
            for (int v = 0; v < 3; ++v) z.simp_col[3 * (f0 + k) + v] = level_id(t[v], J);
          }
        }
      });
    }
  }
}

}  // namespace asmg
