// Host setup of the 3D auxiliary hierarchy (octree; tetrahedral grids).
//
// Closure (Sec. 3.2 in 3D): a split box needs its 6 face and 12 edge
// neighbours of the same depth, so the parents of those neighbours are
// refined one level up, finest depth first.
// Triangulation of a box shown at level l (the 3D counterpart of the
// "closure2" templates): without edge midpoints or subdivided faces, the 6
// Kuhn tetrahedra of its (0,0,0)-(1,1,1) diagonal; otherwise each face --
// subdivided face: its 4 sub-squares split along their min-to-max diagonal;
// face with an edge midpoint: fan about the face centre; other faces: the
// min-to-max diagonal -- coned to the box centre.  Nodes lie on the 2^(J+1)
// lattice of the root cube, named by 63-bit Morton keys; the free nodes of
// the finest level, in key order, are the auxiliary unknowns.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <memory>
#include <thread>
#include <unordered_map>

#include "clip.h"
#include "internal.h"
#include "keyindex.h"

namespace asmg {

namespace {

typedef __int128 i128;

inline uint64_t spread3(uint64_t v) {
  v &= 0x1fffffULL;
  v = (v | (v << 32)) & 0x1f00000000ffffULL;
  v = (v | (v << 16)) & 0x1f0000ff0000ffULL;
  v = (v | (v << 8)) & 0x100f00f00f00f00fULL;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ULL;
  v = (v | (v << 2)) & 0x1249249249249249ULL;
  return v;
}

inline uint64_t compact3(uint64_t v) {
  v &= 0x1249249249249249ULL;
  v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ULL;
  v = (v ^ (v >> 4)) & 0x100f00f00f00f00fULL;
  v = (v ^ (v >> 8)) & 0x1f0000ff0000ffULL;
  v = (v ^ (v >> 16)) & 0x1f00000000ffffULL;
  v = (v ^ (v >> 32)) & 0x1fffffULL;
  return v;
}

inline uint64_t m3(uint64_t x, uint64_t y, uint64_t z) { return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2); }
inline void um3(uint64_t k, uint64_t* q) {
  q[0] = compact3(k);
  q[1] = compact3(k >> 1);
  q[2] = compact3(k >> 2);
}

struct Tree3 {
  int LB = 1;  // lattice bits of auxiliary nodes
  std::vector<std::vector<uint64_t>> S;
  std::vector<KeyIndex> SI;  // lookup tables of S once it is final (index())
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
  bool exists(int d, uint64_t p) const { return d == 0 ? p == 0 : split(d - 1, p >> 3); }
  bool offset(int d, uint64_t p, const int* o, uint64_t& q) const {
    uint64_t c[3];
    um3(p, c);
    const int64_t nb = 1LL << d;
    int64_t n[3];
    for (int k = 0; k < 3; ++k) {
      n[k] = (int64_t)c[k] + o[k];
      if (n[k] < 0 || n[k] >= nb) return false;
    }
    q = m3(n[0], n[1], n[2]);
    return true;
  }
  bool split_at(int d, uint64_t p, int ox, int oy, int oz) const {
    int o[3] = {ox, oy, oz};
    uint64_t q;
    return offset(d, p, o, q) && split(d, q);
  }
};

typedef std::array<uint64_t, 4> Tet;

inline i128 orient(const Tet& t) {
  i128 P[4][3];
  for (int v = 0; v < 4; ++v) {
    uint64_t q[3];
    um3(t[v], q);
    for (int k = 0; k < 3; ++k) P[v][k] = (i128)q[k];
  }
  i128 a[3], b[3], c[3];
  for (int k = 0; k < 3; ++k) {
    a[k] = P[1][k] - P[0][k];
    b[k] = P[2][k] - P[0][k];
    c[k] = P[3][k] - P[0][k];
  }
  return a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) + a[2] * (b[0] * c[1] - b[1] * c[0]);
}

struct BoxShape {
  bool fsub[3][2];     // face subdivided (axis, side)
  bool hang = false;   // any edge midpoint
};

// Is the midpoint of the box edge along axis e, at side sf of axis f and side
// sg of axis g, a node (some other box of that edge is split)?
bool edge_mid(const Tree3& T, int d, uint64_t p, int f, int sf, int g, int sg) {
  int o1[3] = {0, 0, 0}, o2[3] = {0, 0, 0}, o3[3] = {0, 0, 0};
  o1[f] = sf ? 1 : -1;
  o2[g] = sg ? 1 : -1;
  o3[f] = o1[f];
  o3[g] = o2[g];
  return T.split_at(d, p, o1[0], o1[1], o1[2]) || T.split_at(d, p, o2[0], o2[1], o2[2]) ||
         T.split_at(d, p, o3[0], o3[1], o3[2]);
}

BoxShape shape(const Tree3& T, int d, uint64_t p, int lvl) {
  BoxShape s;
  for (int a = 0; a < 3; ++a)
    for (int sd = 0; sd < 2; ++sd) s.fsub[a][sd] = false;
  if (d >= lvl) return s;
  for (int a = 0; a < 3; ++a)
    for (int sd = 0; sd < 2; ++sd) {
      int o[3] = {0, 0, 0};
      o[a] = sd ? 1 : -1;
      s.fsub[a][sd] = T.split_at(d, p, o[0], o[1], o[2]);
    }
  for (int e = 0; e < 3 && !s.hang; ++e) {
    const int f = (e + 1) % 3, g = (e + 2) % 3;
    for (int sf = 0; sf < 2 && !s.hang; ++sf)
      for (int sg = 0; sg < 2 && !s.hang; ++sg)
        if (edge_mid(T, d, p, f, sf, g, sg)) s.hang = true;
  }
  return s;
}

// Tetrahedra of box (d, p) as seen at level lvl; `kuhn` tells which form.
void box_tets(const Tree3& T, int d, uint64_t p, int lvl, std::vector<Tet>& out, bool* kuhn = nullptr) {
  uint64_t c[3];
  um3(p, c);
  const uint64_t s = 1ULL << (T.LB - d), h = s / 2;
  auto pt = [&](int u0, int u1, int u2) { return m3(c[0] * s + u0 * h, c[1] * s + u1 * h, c[2] * s + u2 * h); };
  auto add = [&](Tet t) {
    if (orient(t) < 0) std::swap(t[2], t[3]);
    out.push_back(t);
  };
  BoxShape sh = shape(T, d, p, lvl);
  if (kuhn) *kuhn = !sh.hang;
  if (!sh.hang) {
    static const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (auto& pm : perm) {
      int u1[3] = {0, 0, 0}, u2[3] = {0, 0, 0};
      u1[pm[0]] = 2;
      u2[pm[0]] = 2;
      u2[pm[1]] = 2;
      add({pt(0, 0, 0), pt(u1[0], u1[1], u1[2]), pt(u2[0], u2[1], u2[2]), pt(2, 2, 2)});
    }
    return;
  }
  const uint64_t C = pt(1, 1, 1);
  for (int a = 0; a < 3; ++a) {
    const int b = a == 0 ? 1 : 0, cc = a == 2 ? 1 : 2;
    for (int sd = 0; sd < 2; ++sd) {
      auto fp = [&](int ub, int uc) {
        int u[3];
        u[a] = 2 * sd;
        u[b] = ub;
        u[cc] = uc;
        return pt(u[0], u[1], u[2]);
      };
      if (sh.fsub[a][sd]) {
        for (int sb = 0; sb < 2; ++sb)
          for (int sc = 0; sc < 2; ++sc) {
            add({fp(sb, sc), fp(sb + 1, sc), fp(sb + 1, sc + 1), C});
            add({fp(sb, sc), fp(sb + 1, sc + 1), fp(sb, sc + 1), C});
          }
        continue;
      }
      const bool mc0 = edge_mid(T, d, p, a, sd, cc, 0), mc2 = edge_mid(T, d, p, a, sd, cc, 1);
      const bool mb0 = edge_mid(T, d, p, a, sd, b, 0), mb2 = edge_mid(T, d, p, a, sd, b, 1);
      if (mc0 || mc2 || mb0 || mb2) {
        uint64_t ring[8];
        int n = 0;
        ring[n++] = fp(0, 0);
        if (mc0) ring[n++] = fp(1, 0);
        ring[n++] = fp(2, 0);
        if (mb2) ring[n++] = fp(2, 1);
        ring[n++] = fp(2, 2);
        if (mc2) ring[n++] = fp(1, 2);
        ring[n++] = fp(0, 2);
        if (mb0) ring[n++] = fp(0, 1);
        const uint64_t FC = fp(1, 1);
        for (int i = 0; i < n; ++i) add({ring[i], ring[(i + 1) % n], FC, C});
      } else {
        add({fp(0, 0), fp(2, 0), fp(2, 2), C});
        add({fp(0, 0), fp(2, 2), fp(0, 2), C});
      }
    }
  }
}

inline bool bnd3(const Tree3& T, uint64_t k) {
  uint64_t q[3];
  um3(k, q);
  const uint64_t top = 1ULL << T.LB;
  return q[0] == 0 || q[1] == 0 || q[2] == 0 || q[0] == top || q[1] == top || q[2] == top;
}


void uniq(std::vector<uint64_t>& v) {
  std::sort(v.begin(), v.end());
  v.erase(std::unique(v.begin(), v.end()), v.end());
}

std::vector<uint64_t> boxes_at(const Tree3& T, int d) {
  if (d == 0) return {0};
  std::vector<uint64_t> b;
  if (d - 1 >= (int)T.S.size()) return b;
  b.reserve(T.S[d - 1].size() * 8);
  for (uint64_t p : T.S[d - 1])
    for (uint64_t c = 0; c < 8; ++c) b.push_back((p << 3) | c);
  return b;
}

// ---------------------------------------------------------------- clipping
// A convex region kept as a list of tetrahedra; a plane cut replaces every
// tetrahedron by the tetrahedra of its kept part (0, 1 or 3 pieces).
typedef std::array<double, 3> V3;
typedef std::array<V3, 4> TetP;

inline double vol6(const V3& a, const V3& b, const V3& c, const V3& d) {
  const double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]},
               e3[3] = {d[0] - a[0], d[1] - a[1], d[2] - a[2]};
  return e1[0] * (e2[1] * e3[2] - e2[2] * e3[1]) - e1[1] * (e2[0] * e3[2] - e2[2] * e3[0]) +
         e1[2] * (e2[0] * e3[1] - e2[1] * e3[0]);
}

clip::Tet4 tet4(const TetP& t) {
  clip::Tet4 r;
  for (int v = 0; v < 4; ++v)
    for (int k = 0; k < 3; ++k) r.p[v].v[k] = t[v][k];
  return r;
}

void leaves_in(const Tree3& T, const int64_t* lo, const int64_t* hi, std::vector<std::pair<int, uint64_t>>& out) {
  // depth first; a split box pushes only the children that meet the window,
  // in ascending child order, carrying each box's lattice corner (the depth
  // is at most 20, so at most 7 * 20 + 8 entries are pending)
  struct Ent {
    int d;
    uint64_t p;
    int64_t x[3];
  };
  Ent st[168];
  int top = 0;
  auto meets = [&](int64_t x0, int64_t s, int k) { return !(x0 >= hi[k] || x0 + s <= lo[k]); };
  {
    const int64_t s = 1LL << T.LB;
    if (!(meets(0, s, 0) && meets(0, s, 1) && meets(0, s, 2))) return;
    st[top++] = Ent{0, 0, {0, 0, 0}};
  }
  while (top > 0) {
    const Ent b = st[--top];
    if (!T.split(b.d, b.p)) {
      out.push_back({b.d, b.p});
      continue;
    }
    const int64_t h = 1LL << (T.LB - b.d - 1);
    for (uint64_t ch = 0; ch < 8; ++ch) {
      const int64_t cx = b.x[0] + (int64_t)(ch & 1) * h, cy = b.x[1] + (int64_t)((ch >> 1) & 1) * h,
                    cz = b.x[2] + (int64_t)((ch >> 2) & 1) * h;
      if (meets(cx, h, 0) && meets(cy, h, 1) && meets(cz, h, 2)) st[top++] = Ent{b.d + 1, (b.p << 3) | ch, {cx, cy, cz}};
    }
  }
}

// f(thread, begin, end) over contiguous ranges of [0, n), in thread order
template <class F>
void pfor(int64_t n, F f) {
  unsigned nt = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
  if (n < 2048) nt = 1;
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nt; ++t) th.emplace_back([&, t] { f(t, n * t / nt, n * (t + 1) / nt); });
  for (auto& x : th) x.join();
}

// sorted unique union of per-thread lists (each part deduplicated in
// parallel first)
template <class V>
std::vector<V> uniq_parts(std::vector<std::vector<V>>& parts) {
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

// sort v: contiguous chunks sorted in parallel, then merged pairwise in
// parallel rounds (the result is the sorted sequence, as from std::sort)
template <class V>
void psort(std::vector<V>& v) {
  const int64_t n = (int64_t)v.size();
  unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  if (n < (1 << 16)) nt = 1;
  std::vector<int64_t> cut(nt + 1);
  for (unsigned t = 0; t <= nt; ++t) cut[t] = n * t / nt;
  {
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t) th.emplace_back([&, t] { std::sort(v.begin() + cut[t], v.begin() + cut[t + 1]); });
    for (auto& x : th) x.join();
  }
  for (unsigned w = 1; w < nt; w *= 2) {
    std::vector<std::thread> th;
    for (unsigned t = 0; t + w < nt; t += 2 * w) {
      const int64_t a = cut[t], m = cut[t + w], b = cut[std::min(nt, t + 2 * w)];
      th.emplace_back([&v, a, m, b] { std::inplace_merge(v.begin() + a, v.begin() + m, v.begin() + b); });
    }
    for (auto& x : th) x.join();
  }
}

// index of the Kuhn tetrahedron of a box holding point u (local coordinates
// in units of the box, 0..1): the order of the coordinates
int kuhn_index(const double* u) {
  static const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  for (int k = 0; k < 6; ++k) {
    const int* pm = perm[k];
    if (u[pm[0]] >= u[pm[1]] && u[pm[1]] >= u[pm[2]]) return k;
  }
  return 0;
}

}  // namespace

void lattice_point3(const TreeResult& t, int LB, uint64_t key, double* p) {
  uint64_t q[3];
  um3(key, q);
  for (int k = 0; k < 3; ++k) p[k] = t.amin[k] + std::ldexp((double)q[k], -LB) * t.L;
}

// A fine boundary triangle of Gamma_D (mixed boundaries).
struct GTri {
  double p[3][3];
};

inline void vsub(const double* a, const double* b, double* r) {
  for (int k = 0; k < 3; ++k) r[k] = a[k] - b[k];
}
inline void vcross(const double* a, const double* b, double* r) {
  r[0] = a[1] * b[2] - a[2] * b[1];
  r[1] = a[2] * b[0] - a[0] * b[2];
  r[2] = a[0] * b[1] - a[1] * b[0];
}
inline double vdot(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// The closed triangle g meets the interior of the tetrahedron K exactly when
// no direction separates them, touching allowed.  The directions to try are
// the facet normals of the Minkowski difference K - g: K's face normals, g's
// normal, and the cross products of an edge of K with an edge of g.  With FP64
// projections, an overlap below 1e-12 |a| L along a counts as touching.
inline bool tri_cuts_open_tet(const double K[4][3], const GTri& g, double L) {
  double ax[23][3];
  int na = 0;
  static const int fv[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
  static const int ke[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
  double e1[3], e2[3];
  for (auto& f : fv) {
    vsub(K[f[1]], K[f[0]], e1);
    vsub(K[f[2]], K[f[0]], e2);
    vcross(e1, e2, ax[na++]);
  }
  vsub(g.p[1], g.p[0], e1);
  vsub(g.p[2], g.p[0], e2);
  vcross(e1, e2, ax[na++]);
  for (auto& e : ke)
    for (int t = 0; t < 3; ++t) {
      vsub(K[e[1]], K[e[0]], e1);
      vsub(g.p[(t + 1) % 3], g.p[t], e2);
      vcross(e1, e2, ax[na++]);
    }
  for (int i = 0; i < na; ++i) {
    const double* a = ax[i];
    const double n2 = vdot(a, a);
    if (n2 == 0) continue;
    const double tol = 1e-12 * std::sqrt(n2) * L;
    double k0 = INFINITY, k1 = -INFINITY, t0 = INFINITY, t1 = -INFINITY;
    for (int v = 0; v < 4; ++v) {
      const double d = vdot(a, K[v]);
      k0 = std::min(k0, d);
      k1 = std::max(k1, d);
    }
    for (int v = 0; v < 3; ++v) {
      const double d = vdot(a, g.p[v]);
      t0 = std::min(t0, d);
      t1 = std::max(t1, d);
    }
    if (t1 <= k0 + tol || t0 >= k1 - tol) return false;
  }
  return true;
}

// The point x lies on the closed triangle g (within the same relative 1e-12).
inline bool on_tri(const GTri& g, const double* x, double L) {
  double e1[3], e2[3], n[3], r[3];
  vsub(g.p[1], g.p[0], e1);
  vsub(g.p[2], g.p[0], e2);
  vcross(e1, e2, n);
  const double nn = std::sqrt(vdot(n, n));
  vsub(x, g.p[0], r);
  const double tol = 1e-12 * nn * L;
  if (std::fabs(vdot(n, r)) > tol) return false;
  double s[3];
  for (int k = 0; k < 3; ++k) {
    double a[3], b[3], c[3];
    vsub(g.p[(k + 1) % 3], g.p[k], a);
    vsub(x, g.p[k], b);
    vcross(a, b, c);
    s[k] = vdot(n, c) / nn;
  }
  return (s[0] >= -tol && s[1] >= -tol && s[2] >= -tol) || (s[0] <= tol && s[1] <= tol && s[2] <= tol);
}

// Gamma_D of a mixed problem: the fine boundary faces (faces of one element)
// with three Dirichlet vertices, binned by bounding box on gn^3 cells over
// the root cube.
struct GammaD3 {
  std::vector<GTri> tri;
  int gn = 1;
  double amin[3] = {0, 0, 0}, L = 1;
  std::vector<int64_t> start = std::vector<int64_t>(2, 0);
  std::vector<int32_t> item;

  int cell(double v, int a, double slack) const {
    const double cc = (v - amin[a]) / L * gn + slack;
    return (int)std::min<double>(gn - 1, std::max(0.0, std::floor(cc)));
  }
  void build(const MeshHost& mesh, const TreeResult& tree) {
    for (int a = 0; a < 3; ++a) amin[a] = tree.amin[a];
    L = tree.L;
    std::vector<std::array<int32_t, 3>> fs;
    fs.reserve(4 * mesh.ne);
    for (int64_t e = 0; e < mesh.ne; ++e)
      for (int k = 0; k < 4; ++k) {
        std::array<int32_t, 3> f = {mesh.E[4 * e + (k + 1) % 4], mesh.E[4 * e + (k + 2) % 4], mesh.E[4 * e + (k + 3) % 4]};
        std::sort(f.begin(), f.end());
        fs.push_back(f);
      }
    std::sort(fs.begin(), fs.end());
    for (size_t i = 0; i < fs.size();) {
      size_t j = i;
      while (j < fs.size() && fs[j] == fs[i]) ++j;
      if (j - i == 1 && mesh.bflag[fs[i][0]] == 1 && mesh.bflag[fs[i][1]] == 1 && mesh.bflag[fs[i][2]] == 1) {
        GTri g;
        for (int v = 0; v < 3; ++v)
          for (int k = 0; k < 3; ++k) g.p[v][k] = mesh.X[3 * (int64_t)fs[i][v] + k];
        tri.push_back(g);
      }
      i = j;
    }
    gn = std::max(1, std::min(128, (int)std::cbrt((double)tri.size())));
    start.assign((size_t)gn * gn * gn + 1, 0);
    for (int pass = 0; pass < 2; ++pass) {
      std::vector<int64_t> fill(start.begin(), start.end() - 1);
      for (size_t q = 0; q < tri.size(); ++q) {
        int c0[3], c1[3];
        for (int a = 0; a < 3; ++a) {
          c0[a] = cell(std::min({tri[q].p[0][a], tri[q].p[1][a], tri[q].p[2][a]}), a, -1e-9);
          c1[a] = cell(std::max({tri[q].p[0][a], tri[q].p[1][a], tri[q].p[2][a]}), a, 1e-9);
        }
        for (int z = c0[2]; z <= c1[2]; ++z)
          for (int y = c0[1]; y <= c1[1]; ++y)
            for (int x = c0[0]; x <= c1[0]; ++x) {
              const int64_t ci = ((int64_t)z * gn + y) * gn + x;
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
  // f(triangle) for the triangles binned in the cells the box [lo, hi]
  // meets; stops when f returns true
  template <class F>
  bool any(const double* lo, const double* hi, F&& f) const {
    int c0[3], c1[3];
    for (int a = 0; a < 3; ++a) {
      c0[a] = cell(lo[a], a, -1e-9);
      c1[a] = cell(hi[a], a, 1e-9);
    }
    for (int z = c0[2]; z <= c1[2]; ++z)
      for (int y = c0[1]; y <= c1[1]; ++y)
        for (int x = c0[0]; x <= c1[0]; ++x) {
          const int64_t ci = ((int64_t)z * gn + y) * gn + x;
          for (int64_t q = start[ci]; q < start[ci + 1]; ++q)
            if (f(tri[item[q]])) return true;
        }
    return false;
  }
  // the interior of the tetrahedron K meets Gamma_D
  bool cuts(const double K[4][3]) const {
    if (tri.empty()) return false;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int v = 0; v < 4; ++v)
      for (int a = 0; a < 3; ++a) {
        lo[a] = std::min(lo[a], K[v][a]);
        hi[a] = std::max(hi[a], K[v][a]);
      }
    return any(lo, hi, [&](const GTri& g) { return tri_cuts_open_tet(K, g, L); });
  }
  // the point P lies on Gamma_D
  bool on(const double* P) const {
    if (tri.empty()) return false;
    return any(P, P, [&](const GTri& g) { return on_tri(g, P, L); });
  }
};

void build_aux_host3(const MeshHost& mesh, const TreeResult& tree, const asmg_params& prm, AuxHost& out) {
  // R18: a Neumann vertex selects the mixed grids (tetrahedra whose interior
  // meets Omega and no Gamma_D triangle)
  const bool mixed = mesh.mixed;
  Tree3 T;
  T.S = tree.split;
  // closure, finest depth first: the parents of all face and edge neighbours
  // of every split box are split
  for (int d = (int)T.S.size() - 1; d >= 1; --d) {
    std::vector<uint64_t> add;
    for (uint64_t p : T.S[d])
      for (int oz = -1; oz <= 1; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
          for (int ox = -1; ox <= 1; ++ox) {
            const int nz = (ox != 0) + (oy != 0) + (oz != 0);
            if (nz < 1 || nz > 2) continue;
            int o[3] = {ox, oy, oz};
            uint64_t q;
            if (T.offset(d, p, o, q)) add.push_back(q >> 3);
          }
    auto& up = T.S[d - 1];
    up.insert(up.end(), add.begin(), add.end());
    uniq(up);
  }
  out.split = T.S;
  const int J = (int)T.S.size();
  out.J = J;
  if (J + 1 > 21) ASMG_FAIL(ASMG_ERR_UNSUPPORTED, "3D auxiliary hierarchy deeper than 20 levels");
  T.LB = J + 1;
  out.LB = T.LB;
  T.index();
  std::vector<std::vector<uint64_t>> BX(J + 1);
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

  // finest-level free nodes: the non-boundary vertices of the leaves'
  // tetrahedra
  {
    std::vector<std::pair<int, uint64_t>> leaves;
    for (int d = 0; d <= J; ++d)
      for (uint64_t p : BX[d])
        if (!T.split(d, p)) leaves.push_back({d, p});
    const unsigned nt = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
    std::vector<std::vector<uint64_t>> part(nt);
    pfor((int64_t)leaves.size(), [&](unsigned t, int64_t b0, int64_t b1) {
      std::vector<Tet> tt;
      for (int64_t q = b0; q < b1; ++q) {
        tt.clear();
        box_tets(T, leaves[q].first, leaves[q].second, J, tt);
        for (auto& x : tt)
          for (int k = 0; k < 4; ++k)
            if (mixed || !bnd3(T, x[k])) part[t].push_back(x[k]);
      }
    });
    out.aux_key = uniq_parts(part);
  }
  const std::vector<uint64_t>& AK = out.aux_key;

  // per level: changed boxes at depth l-1, new nodes and their two parents
  out.nlevel.assign(J + 1, 0);
  std::vector<std::vector<uint64_t>> changed(J + 1);
  std::vector<std::vector<std::array<uint64_t, 3>>> newnodes(J + 1);
  for (int l = 1; l <= J; ++l) {
    const int d = l - 1;
    const uint64_t s = 1ULL << (T.LB - d), h = s / 2;
    // per-thread runs of consecutive boxes, appended in box order
    const unsigned ntn = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
    std::vector<std::vector<std::array<uint64_t, 3>>> nparts(ntn);
    std::vector<std::vector<uint64_t>> cparts(ntn);
    pfor((int64_t)BX[d].size(), [&](unsigned tix, int64_t b0, int64_t b1) {
    auto& nn = nparts[tix];
    for (int64_t bi = b0; bi < b1; ++bi) {
      const uint64_t p = BX[d][bi];
      const bool sp = T.split(d, p);
      BoxShape sh = shape(T, d, p, l);
      if (!sp && !sh.hang) continue;
      cparts[tix].push_back(p);
      uint64_t c[3];
      um3(p, c);
      auto pt = [&](int u0, int u1, int u2) { return m3(c[0] * s + u0 * h, c[1] * s + u1 * h, c[2] * s + u2 * h); };
      nn.push_back({pt(1, 1, 1), pt(0, 0, 0), pt(2, 2, 2)});  // centre: midpoint of the main diagonal
      for (int a = 0; a < 3; ++a) {
        const int b = a == 0 ? 1 : 0, cc = a == 2 ? 1 : 2;
        for (int sd = 0; sd < 2; ++sd) {
          auto fp = [&](int ub, int uc) {
            int u[3];
            u[a] = 2 * sd;
            u[b] = ub;
            u[cc] = uc;
            return pt(u[0], u[1], u[2]);
          };
          // face centre (midpoint of the face's min-to-max diagonal) is a node
          // of split boxes and of fanned or subdivided faces
          bool fan = sp || sh.fsub[a][sd] || edge_mid(T, d, p, a, sd, cc, 0) || edge_mid(T, d, p, a, sd, cc, 1) ||
                     edge_mid(T, d, p, a, sd, b, 0) || edge_mid(T, d, p, a, sd, b, 1);
          if (fan) nn.push_back({fp(1, 1), fp(0, 0), fp(2, 2)});
        }
      }
      if (sp)
        for (int e = 0; e < 3; ++e) {
          const int f = (e + 1) % 3, g = (e + 2) % 3;
          for (int sf = 0; sf < 2; ++sf)
            for (int sg = 0; sg < 2; ++sg) {
              int u0[3], u1[3], um[3];
              u0[e] = 0;
              u1[e] = 2;
              um[e] = 1;
              u0[f] = u1[f] = um[f] = 2 * sf;
              u0[g] = u1[g] = um[g] = 2 * sg;
              nn.push_back({pt(um[0], um[1], um[2]), pt(u0[0], u0[1], u0[2]), pt(u1[0], u1[1], u1[2])});
            }
        }
    }
    });
    std::vector<std::array<uint64_t, 3>> nn;
    for (unsigned t = 0; t < ntn; ++t) {
      nn.insert(nn.end(), nparts[t].begin(), nparts[t].end());
      changed[l].insert(changed[l].end(), cparts[t].begin(), cparts[t].end());
    }
    std::sort(nn.begin(), nn.end());
    nn.erase(std::unique(nn.begin(), nn.end(),
                         [](const std::array<uint64_t, 3>& x, const std::array<uint64_t, 3>& y) { return x[0] == y[0]; }),
             nn.end());
    int64_t nf = 0;
    for (auto& v : nn)
      if (!bnd3(T, v[0])) ++nf;
    out.nlevel[l] = out.nlevel[l - 1] + nf;
    newnodes[l] = std::move(nn);
  }
  // tetrahedra of every leaf box at the finest level: ftet[first[d][i] ..
  // first[d][i] + nft[d][i]) for leaf i of depth d (first = -1: split box)
  std::vector<Tet> ftet;
  std::vector<std::vector<int64_t>> first(J + 1);
  std::vector<std::vector<uint8_t>> nft(J + 1);
  std::vector<std::vector<int32_t>> lid(J + 1);  // leaf number
  int64_t nleaf = 0;
  for (int d = 0; d <= J; ++d) {
    first[d].assign(BX[d].size(), -1);
    nft[d].assign(BX[d].size(), 0);
    lid[d].assign(BX[d].size(), -1);
    // per-thread runs of consecutive boxes, appended in box order
    const unsigned ntl = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
    std::vector<std::vector<Tet>> tparts(ntl);
    std::vector<uint8_t> isleaf(BX[d].size(), 0);
    pfor((int64_t)BX[d].size(), [&](unsigned t, int64_t b0, int64_t b1) {
      for (int64_t i = b0; i < b1; ++i) {
        if (T.split(d, BX[d][i])) continue;
        isleaf[i] = 1;
        const size_t before = tparts[t].size();
        box_tets(T, d, BX[d][i], J, tparts[t]);
        nft[d][i] = (uint8_t)(tparts[t].size() - before);
      }
    });
    const int64_t base = (int64_t)ftet.size();
    int64_t at = base;
    for (size_t i = 0; i < BX[d].size(); ++i) {
      if (!isleaf[i]) continue;
      first[d][i] = at;
      lid[d][i] = (int32_t)nleaf++;
      at += nft[d][i];
    }
    ftet.resize(at);
    int64_t pos = base;
    for (auto& tp : tparts) {
      std::copy(tp.begin(), tp.end(), ftet.begin() + pos);
      pos += (int64_t)tp.size();
    }
  }
  const double lat_scale = std::ldexp(1.0, T.LB) / tree.L;
  // lattice window holding a fine tetrahedron's bounding box (widened by
  // 1e-9 lattice units against rounding of the scaling)
  auto window = [&](const TetP& S, int64_t* lo, int64_t* hi) {
    for (int k = 0; k < 3; ++k) {
      double mn = S[0][k], mx = S[0][k];
      for (int v = 1; v < 4; ++v) {
        mn = std::min(mn, S[v][k]);
        mx = std::max(mx, S[v][k]);
      }
      lo[k] = (int64_t)std::floor((mn - tree.amin[k]) * lat_scale - 1e-9);
      hi[k] = (int64_t)std::ceil((mx - tree.amin[k]) * lat_scale + 1e-9);
    }
  };
  auto fine_tet = [&](int64_t e, TetP& S) {
    for (int v = 0; v < 4; ++v)
      for (int k = 0; k < 3; ++k) S[v][k] = mesh.X[(int64_t)mesh.E[4 * e + v] * 3 + k];
  };
  auto leaf_tet = [&](int64_t q, TetP& K) {
    for (int v = 0; v < 4; ++v) lattice_point3(tree, T.LB, ftet[q][v], K[v].data());
  };
  auto leaf_range = [&](const std::pair<int, uint64_t>& lf, int64_t& f0, int& nq, int32_t* leaf = nullptr) {
    const size_t bi = box_at(lf.first, lf.second);
    f0 = first[lf.first][bi];
    nq = nft[lf.first][bi];
    if (leaf) *leaf = lid[lf.first][bi];
  };

  // element coefficients: integrals of a over the 6 Kuhn tetrahedra of every
  // box (bottom-up) and over the fan tetrahedra of fanned leaves
  const bool varcoef = !mesh.coeff.empty();
  // R17: a domain that does not fill the root cube uses the Dirichlet grids
  // T^D_l (tetrahedra inside Omega); the clipping pass then also measures how
  // much of each tetrahedron the fine elements cover (kcov, fancov)
  const bool dgrid = !mesh.boxdomain && !mixed;
  const bool cover = dgrid || mixed;  // the clipping pass also measures covered volumes
  std::vector<std::vector<std::array<double, 6>>> kint(J + 1), kcov(J + 1);
  std::unordered_map<uint64_t, double> fanint, fancov;  // keyed by the sorted tet's hash below
  auto tet_hash = [](Tet t) {
    std::sort(t.begin(), t.end());
    uint64_t hsh = 1469598103934665603ULL;
    for (auto v : t) hsh = (hsh ^ v) * 1099511628211ULL;
    return hsh;
  };
  if (varcoef || cover) {
    // the constant-leaf shortcut below needs elements that tile every leaf
    const bool skip_const = varcoef && !cover;
    // elements in Morton order of their lowest corner, in chunks of 4096;
    // each chunk sums its overlaps per leaf tetrahedron, and the chunk sums
    // are added in chunk order (deterministic for any thread count)
    std::vector<std::pair<uint64_t, int32_t>> order(mesh.ne);
    pfor(mesh.ne, [&](unsigned, int64_t b0, int64_t b1) {
      for (int64_t e = b0; e < b1; ++e) {
        TetP S;
        fine_tet(e, S);
        uint64_t q[3];
        for (int k = 0; k < 3; ++k) {
          double mn = std::min(std::min(S[0][k], S[1][k]), std::min(S[2][k], S[3][k]));
          double u = std::floor((mn - tree.amin[k]) * lat_scale);
          q[k] = (uint64_t)std::min(std::max(u, 0.0), std::ldexp(1.0, T.LB) - 1);
        }
        order[e] = {m3(q[0], q[1], q[2]), (int32_t)e};
      }
    });
    psort(order);
    const int64_t CH = 4096, nch = (mesh.ne + CH - 1) / CH;
    // A leaf whose overlapping elements all have one coefficient value a has
    // the average a on each of its tetrahedra (the fine elements tile it): only
    // leaves that see two values are clipped.  The elements whose bounding
    // boxes meet a leaf include every element that overlaps it.  Per leaf:
    // the bits of the first value seen (0: none yet) and a "mixed" flag.
    // A leaf that sees two values keeps the smallest bit pattern seen, a0
    // (deterministic for any thread count): since the elements tile it,
    // int_K a = a0 |K| + sum_e (a_e - a0) |e n K|, and only its elements with
    // a_e != a0 are clipped.
    std::vector<std::atomic<uint64_t>> lval(nleaf), lmin(nleaf);
    std::vector<std::atomic<uint8_t>> lmixed(nleaf);
    for (int64_t q = 0; q < nleaf; ++q) {
      lval[q].store(0, std::memory_order_relaxed);
      lmin[q].store(~0ULL, std::memory_order_relaxed);
      lmixed[q].store(0, std::memory_order_relaxed);
    }
    // The leaves each element meets are kept from this pass for the clipping
    // pass (CSR over the elements in Morton order, each list in the order
    // leaves_in gives it), with every leaf's first finest tetrahedron and
    // count.  Morton order keeps the tree lookups of neighbouring elements
    // close together.
    std::vector<int64_t> eoff, lf0(nleaf, 0);
    std::vector<int32_t> eleaf, lnq(nleaf, 0);
    std::vector<std::vector<int32_t>> tl(64);
    std::vector<int64_t> tb0(64, -1);
    std::vector<uint32_t> ecnt;
    if (skip_const) {
      for (int d = 0; d <= J; ++d)
        for (size_t i = 0; i < BX[d].size(); ++i)
          if (lid[d][i] >= 0) {
            lf0[lid[d][i]] = first[d][i];
            lnq[lid[d][i]] = nft[d][i];
          }
      ecnt.assign(mesh.ne, 0);
    }
    if (skip_const) pfor(mesh.ne, [&](unsigned t, int64_t b0, int64_t b1) {
      std::vector<std::pair<int, uint64_t>> lv;
      tb0[t] = b0;
      // the last leaves looked up (elements in Morton order share most of theirs)
      struct Hit {
        int d = -1;
        uint64_t p = 0;
        int32_t leaf = -1;
      } cache[16];
      for (int64_t k = b0; k < b1; ++k) {
        const int64_t e = order[k].second;
        TetP S;
        fine_tet(e, S);
        int64_t lo[3], hi[3];
        window(S, lo, hi);
        lv.clear();
        leaves_in(T, lo, hi, lv);
        uint64_t bits;
        std::memcpy(&bits, &mesh.coeff[e], 8);
        ecnt[k] = (uint32_t)lv.size();
        for (auto& lf : lv) {
          Hit& hc = cache[(lf.second ^ (uint64_t)lf.first * 0x9E3779B97F4A7C15ULL) & 15];
          if (hc.d != lf.first || hc.p != lf.second) {
            int64_t f0;
            int nq;
            leaf_range(lf, f0, nq, &hc.leaf);
            hc.d = lf.first;
            hc.p = lf.second;
          }
          const int32_t leaf = hc.leaf;
          tl[t].push_back(leaf);
          // first value seen, else a second one makes the leaf mixed (an atomic
          // write only while the leaf is still empty or not yet mixed)
          uint64_t expect = lval[leaf].load(std::memory_order_relaxed);
          if (expect == 0 && lval[leaf].compare_exchange_strong(expect, bits, std::memory_order_relaxed)) expect = bits;
          if (expect != bits && !lmixed[leaf].load(std::memory_order_relaxed))
            lmixed[leaf].store(1, std::memory_order_relaxed);
          uint64_t cur = lmin[leaf].load(std::memory_order_relaxed);
          while (bits < cur && !lmin[leaf].compare_exchange_weak(cur, bits, std::memory_order_relaxed)) {
          }
        }
      }
    });
    if (skip_const) {
      eoff.assign(mesh.ne + 1, 0);
      for (int64_t e = 0; e < mesh.ne; ++e) eoff[e + 1] = eoff[e] + ecnt[e];
      eleaf.resize(eoff[mesh.ne]);
      std::vector<std::thread> th;
      for (int t = 0; t < 64; ++t) {
        if (tb0[t] < 0 || tl[t].empty()) continue;
        th.emplace_back([&, t] { std::copy(tl[t].begin(), tl[t].end(), eleaf.begin() + eoff[tb0[t]]); });
      }
      for (auto& x : th) x.join();
      std::vector<std::vector<int32_t>>().swap(tl);
      std::vector<uint32_t>().swap(ecnt);
    }
    std::vector<std::vector<std::pair<int64_t, double>>> csum(nch), ccov(nch);
    std::atomic<int64_t> nextc(0);
    auto work = [&]() {
      std::vector<std::pair<int, uint64_t>> lv;
      std::vector<std::pair<int64_t, double>> acc, cac;
      for (;;) {
        const int64_t ch = nextc.fetch_add(1);
        if (ch >= nch) return;
        acc.clear();
        cac.clear();
        for (int64_t k = ch * CH; k < std::min(mesh.ne, (ch + 1) * CH); ++k) {
          const int64_t e = order[k].second;
          TetP S;
          fine_tet(e, S);
          int64_t nl;
          if (skip_const) {
            nl = eoff[k + 1] - eoff[k];
          } else {
            int64_t lo[3], hi[3];
            window(S, lo, hi);
            lv.clear();
            leaves_in(T, lo, hi, lv);
            nl = (int64_t)lv.size();
          }
          for (int64_t r = 0; r < nl; ++r) {
            int64_t f0;
            int nq;
            int32_t leaf;
            if (skip_const) {
              leaf = eleaf[eoff[k] + r];
              f0 = lf0[leaf];
              nq = lnq[leaf];
            } else {
              leaf_range(lv[r], f0, nq, &leaf);
            }
            double a0 = 0;  // mixed leaf: the part a0 |K| is added after the sums
            if (skip_const) {
              if (!lmixed[leaf].load(std::memory_order_relaxed) && lval[leaf].load(std::memory_order_relaxed) != 0)
                continue;
              const uint64_t mb = lmin[leaf].load(std::memory_order_relaxed);
              uint64_t bits;
              std::memcpy(&bits, &mesh.coeff[e], 8);
              if (bits == mb) continue;
              std::memcpy(&a0, &mb, 8);
            }
            for (int q = 0; q < nq; ++q) {
              TetP K;
              leaf_tet(f0 + q, K);
              double vol = 0;
              clip::clip_tets(tet4(S), tet4(K), [&](const clip::Tet4& pc) { vol += clip::volume(pc); });
              if (!(vol > 0)) continue;
              if (varcoef) acc.push_back({f0 + q, vol * (mesh.coeff[e] - a0)});
              if (cover) cac.push_back({f0 + q, vol});
            }
          }
        }
        auto reduce = [](std::vector<std::pair<int64_t, double>>& a, std::vector<std::pair<int64_t, double>>& out) {
          std::stable_sort(a.begin(), a.end(), [](const std::pair<int64_t, double>& x,
                                                  const std::pair<int64_t, double>& y) { return x.first < y.first; });
          for (size_t i = 0; i < a.size();) {
            size_t j = i;
            double sum = 0;
            while (j < a.size() && a[j].first == a[i].first) sum += a[j++].second;
            out.push_back({a[i].first, sum});
            i = j;
          }
        };
        reduce(acc, csum[ch]);
        reduce(cac, ccov[ch]);
      }
    };
    {
      unsigned nt = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
      std::vector<std::thread> th;
      for (unsigned t = 0; t < nt; ++t) th.emplace_back(work);
      for (auto& x : th) x.join();
    }
    std::vector<double> I(ftet.size(), 0.0), C(ftet.size(), 0.0);
    for (auto& v : csum)
      for (auto& pr : v) I[pr.first] += pr.second;
    for (auto& v : ccov)
      for (auto& pr : v) C[pr.first] += pr.second;
    csum.clear();
    ccov.clear();
    if (skip_const)
    for (int d = 0; d <= J; ++d)
      for (size_t i = 0; i < BX[d].size(); ++i) {
        const int32_t leaf = lid[d][i];
        if (leaf < 0 || lval[leaf].load() == 0) continue;
        const bool mixedleaf = lmixed[leaf].load() != 0;
        const uint64_t bits = mixedleaf ? lmin[leaf].load() : lval[leaf].load();
        double a;
        std::memcpy(&a, &bits, 8);
        for (int q = 0; q < nft[d][i]; ++q) {
          TetP K;
          leaf_tet(first[d][i] + q, K);
          const double part = a * (std::fabs(vol6(K[0], K[1], K[2], K[3])) / 6.0);
          I[first[d][i] + q] = mixedleaf ? I[first[d][i] + q] + part : part;
        }
      }
    // bottom-up Kuhn integrals: a (kint, fanint) and the covered volume
    // (kcov, fancov)
    for (int pass = 0; pass < 2; ++pass) {
    if (pass == 0 && !varcoef) continue;
    if (pass == 1 && !cover) continue;
    const std::vector<double>& IA = pass == 0 ? I : C;
    auto& KI = pass == 0 ? kint : kcov;
    auto& FI = pass == 0 ? fanint : fancov;
    for (int d = J; d >= 0; --d) {
      KI[d].assign(BX[d].size(), {0, 0, 0, 0, 0, 0});
      const uint64_t s = 1ULL << (T.LB - d);
      const unsigned ntb = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
      std::vector<std::vector<std::pair<uint64_t, double>>> fparts(ntb);
      pfor((int64_t)BX[d].size(), [&](unsigned tix, int64_t i0, int64_t i1) {
      for (int64_t i = i0; i < i1; ++i) {
        const uint64_t p = BX[d][i];
        uint64_t cb[3];
        um3(p, cb);
        auto local_kuhn = [&](const Tet& t) {  // Kuhn index of t's centroid in this box
          double u[3] = {0, 0, 0};
          for (int v = 0; v < 4; ++v) {
            uint64_t q[3];
            um3(t[v], q);
            for (int k = 0; k < 3; ++k) u[k] += ((double)q[k] - (double)(cb[k] * s)) / (4.0 * (double)s);
          }
          return kuhn_index(u);
        };
        if (!T.split(d, p)) {
          const int64_t f0 = first[d][i];
          const int nq = nft[d][i];
          const bool kuhn = nq == 6;  // a coned box has at least 12 tetrahedra
          for (int q = 0; q < nq; ++q) {
            KI[d][i][local_kuhn(ftet[f0 + q])] += IA[f0 + q];
            if (!kuhn) fparts[tix].push_back({tet_hash(ftet[f0 + q]), IA[f0 + q]});
          }
        } else {
          const auto& ch = BX[d + 1];
          const size_t j = box_at(d + 1, p << 3);
          for (int cidx = 0; cidx < 8; ++cidx) {
            const uint64_t cp = ch[j + cidx];
            std::vector<Tet> kt;
            box_tets(T, d + 1, cp, d + 1, kt);  // the child's 6 Kuhn tetrahedra
            for (int q = 0; q < 6; ++q) KI[d][i][local_kuhn(kt[q])] += KI[d + 1][j + cidx][q];
          }
        }
      }
      });
      for (auto& fp : fparts)
        for (auto& kv : fp) FI[kv.first] = kv.second;
    }
    }
  }
  // tetrahedron q of box (d, p) at a level where the box shows as Kuhn
  // (kuhn) or coned: in T^D_l when the fine elements cover (1 - 1e-9) of it
  auto tet_vol = [&](const Tet& t) {
    double P[4][3];
    for (int v = 0; v < 4; ++v) lattice_point3(tree, T.LB, t[v], P[v]);
    V3 a = {P[0][0], P[0][1], P[0][2]}, b = {P[1][0], P[1][1], P[1][2]}, cc = {P[2][0], P[2][1], P[2][2]},
       dd = {P[3][0], P[3][1], P[3][2]};
    return std::fabs(vol6(a, b, cc, dd)) / 6.0;
  };
  auto tet_cov = [&](int d, uint64_t p, bool kuhn, int q, const Tet& t) -> double {
    if (kuhn) return kcov[d][box_at(d, p)][q];
    auto it = fancov.find(tet_hash(t));
    return it == fancov.end() ? 0.0 : it->second;
  };
  // Gamma_D (mixed): the interior of lattice tetrahedron t meets it; lattice
  // node x lies on it
  GammaD3 gdl;
  if (mixed) gdl.build(mesh, tree);
  auto gd_cuts = [&](const Tet& t) -> bool {
    double K[4][3];
    for (int v = 0; v < 4; ++v) lattice_point3(tree, T.LB, t[v], K[v]);
    return gdl.cuts(K);
  };
  auto on_gd = [&](uint64_t x) -> bool {
    double P[3];
    lattice_point3(tree, T.LB, x, P);
    return gdl.on(P);
  };
  auto tet_inside = [&](int d, uint64_t p, bool kuhn, int q, const Tet& t) -> bool {
    if (mixed) return tet_cov(d, p, kuhn, q, t) > 1e-12 * tet_vol(t) && !gd_cuts(t);
    if (!dgrid) return true;
    return tet_cov(d, p, kuhn, q, t) >= (1.0 - 1e-9) * tet_vol(t);
  };
  // node x is free at level l (a vertex of sigma^(l) off the boundary of
  // Omega^D_l): every level-l tetrahedron around it is inside.  The box
  // shown at level l around x in each octant holds those tetrahedra.
  // Mixed: x is free when it is a node of a kept tetrahedron, lies on no
  // tetrahedron cut by Gamma_D and not on Gamma_D itself.
  auto free_at = [&](uint64_t x, int l, std::vector<Tet>& kt) -> bool {
    if (!mixed && bnd3(T, x)) return false;
    uint64_t X[3];
    um3(x, X);
    bool node = false;
    for (int oct = 0; oct < 8; ++oct) {
      int d = 0;
      uint64_t p = 0;
      while (d < l && T.split(d, p)) {
        const uint64_t sz = 1ULL << (T.LB - d), hf = sz >> 1;
        uint64_t cb[3], ch = 0;
        um3(p, cb);
        for (int a = 0; a < 3; ++a) {
          const uint64_t x0 = cb[a] * sz;
          const bool pos = (oct >> a) & 1;
          const uint64_t bit = pos ? (X[a] >= x0 + hf) : (X[a] > x0 + hf);
          ch |= bit << a;
        }
        p = (p << 3) | ch;
        ++d;
      }
      kt.clear();
      bool kuhn = false;
      box_tets(T, d, p, l, kt, &kuhn);
      for (size_t q = 0; q < kt.size(); ++q) {
        if (kt[q][0] != x && kt[q][1] != x && kt[q][2] != x && kt[q][3] != x) continue;
        if (mixed) {
          if (gd_cuts(kt[q])) return false;
          if (tet_cov(d, p, kuhn, (int)q, kt[q]) > 1e-12 * tet_vol(kt[q])) node = true;
          continue;
        }
        node = true;
        if (!tet_inside(d, p, kuhn, (int)q, kt[q])) return false;
      }
    }
    return node && !(mixed && on_gd(x));
  };
  std::vector<int32_t> phi;  // first level at which each aux node is free (Dirichlet and mixed grids)
  std::vector<int32_t> psi;  // mixed: first level after phi at which it is no longer free
  if (mixed) {
    std::vector<std::pair<uint64_t, int32_t>> born;
    for (int l = 1; l <= J; ++l)
      for (auto& v : newnodes[l]) born.push_back({v[0], l});
    std::sort(born.begin(), born.end());
    const std::vector<uint64_t> cand = out.aux_key;
    std::vector<int32_t> cphi(cand.size(), J + 1), cpsi(cand.size(), J + 1);
    pfor((int64_t)cand.size(), [&](unsigned, int64_t b0, int64_t b1) {
      std::vector<Tet> kt;
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
    std::vector<int32_t> keep(out.aux_key.size(), 0);
    pfor((int64_t)out.aux_key.size(), [&](unsigned, int64_t b0, int64_t b1) {
      std::vector<Tet> kt;
      for (int64_t q = b0; q < b1; ++q) keep[q] = free_at(out.aux_key[q], J, kt);
    });
    std::vector<uint64_t> ak;
    for (size_t q = 0; q < keep.size(); ++q)
      if (keep[q]) ak.push_back(out.aux_key[q]);
    out.aux_key.swap(ak);
    // from its birth level on, a node is free from the first level whose
    // tetrahedra around it are all inside (they only shrink inside covered ones)
    std::vector<std::pair<uint64_t, int32_t>> born;
    for (int l = 1; l <= J; ++l)
      for (auto& v : newnodes[l]) born.push_back({v[0], l});
    std::sort(born.begin(), born.end());
    phi.assign(AK.size(), J + 1);
    pfor((int64_t)AK.size(), [&](unsigned, int64_t b0, int64_t b1) {
      std::vector<Tet> kt;
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
    if (bnd3(T, x)) return -1;
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

  // mean of a over the tetrahedron (a = 0 outside Omega, a = 1 inside when no
  // coefficient is given)
  auto tet_coef = [&](int d, uint64_t p, bool kuhn, int q, const Tet& t) -> double {
    if (mixed) {
      // the mean of a over tau n Omega (R18)
      if (!varcoef) return 1.0;
      const double in = kuhn ? kint[d][box_at(d, p)][q] : fanint.at(tet_hash(t));
      return in / tet_cov(d, p, kuhn, q, t);
    }
    if (!varcoef && !dgrid) return 1.0;
    const auto& KI = varcoef ? kint : kcov;
    const auto& FI = varcoef ? fanint : fancov;
    double P[4][3];
    for (int v = 0; v < 4; ++v) lattice_point3(tree, T.LB, t[v], P[v]);
    V3 a = {P[0][0], P[0][1], P[0][2]}, b = {P[1][0], P[1][1], P[1][2]}, cc = {P[2][0], P[2][1], P[2][2]},
       dd = {P[3][0], P[3][1], P[3][2]};
    const double vol = std::fabs(vol6(a, b, cc, dd)) / 6.0;
    if (kuhn) {
      const size_t i = box_at(d, p);
      return KI[d][i][q] / vol;
    }
    return FI.at(tet_hash(t)) / vol;
  };

  auto emit_box = [&](int d, uint64_t p, int l, std::vector<int32_t>& ids, std::vector<uint64_t>& keys,
                      std::vector<double>& coef, std::vector<Tet>& kt) {  // kt: the caller's scratch
    kt.clear();
    bool kuhn = false;
    box_tets(T, d, p, l, kt, &kuhn);
    for (size_t q = 0; q < kt.size(); ++q) {
      if (!tet_inside(d, p, kuhn, (int)q, kt[q])) continue;  // outside Omega: not in T^D_l
      for (int v = 0; v < 4; ++v) {
        keys.push_back(kt[q][v]);
        ids.push_back(level_id(kt[q][v], l));
      }
      coef.push_back(tet_coef(d, p, kuhn, (int)q, kt[q]));
    }
  };

  // coarsest level
  std::vector<Tet> ckt;  // scratch
  for (int d = 0; d <= c; ++d)
    for (uint64_t p : BX[d]) {
      if (d < c && T.split(d, p)) continue;
      emit_box(d, p, c, out.coarse_tri_id, out.coarse_tri_key, out.coarse_tri_coef, ckt);
    }
  for (auto id : out.coarse_tri_id)
    if (id >= 0) out.coarse_id.push_back(id);
  std::sort(out.coarse_id.begin(), out.coarse_id.end());
  out.coarse_id.erase(std::unique(out.coarse_id.begin(), out.coarse_id.end()), out.coarse_id.end());

  // levels c+1..J, each in parallel over its changed boxes: relevant boxes
  // and smoothing nodes per chunk (merged, sorted, unique), then the level
  // tetrahedra per chunk of relevant boxes, concatenated in order
  out.levels.assign(std::max(0, J - c), AuxLevelHost());
  unsigned nthr = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
  // local smoothing: smoothing nodes (by aux ID) and relevant boxes (by index
  // within their depth) of one level are marked in flag arrays and gathered
  // in ascending order; the flags are cleared for the next level
  const bool local = prm.smoothing != 1 && !mixed;  // the mixed grids are not nested: whole levels
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
    std::vector<std::pair<int, uint64_t>> rel;
    std::vector<uint64_t> sm;
    if (!local) {
      for (int dd = 0; dd <= l; ++dd)
        for (uint64_t p : BX[dd])
          if (!(dd < l && T.split(dd, p))) rel.push_back({dd, p});
      std::vector<std::vector<uint64_t>> part(nthr);
      pfor((int64_t)rel.size(), [&](unsigned t, int64_t b0, int64_t b1) {
        std::vector<Tet> kt;
        for (int64_t q = b0; q < b1; ++q) {
          kt.clear();
          box_tets(T, rel[q].first, rel[q].second, l, kt);
          for (auto& tt : kt)
            for (int v = 0; v < 4; ++v)
              if (level_id(tt[v], l) >= 0) part[t].push_back(tt[v]);
        }
      });
      sm = uniq_parts(part);
    } else {
      const std::vector<uint64_t>& ch = changed[l];
      auto mark_node = [&](int32_t id) {
        if (id >= 0) sflag[id].store(1, std::memory_order_relaxed);
      };
      auto mark_box = [&](int dd, uint64_t pp) {
        rflag[dd][box_at(dd, pp)].store(1, std::memory_order_relaxed);
      };
      pfor((int64_t)ch.size(), [&](unsigned, int64_t b0, int64_t b1) {
        std::vector<Tet> kt;
        for (int64_t q = b0; q < b1; ++q) {
          const uint64_t p = ch[q];
          // free vertices of the box's new tetrahedra (inside Omega)
          auto add = [&](int dd, uint64_t pp) {
            kt.clear();
            bool kuhn = false;
            box_tets(T, dd, pp, l, kt, &kuhn);
            for (size_t k = 0; k < kt.size(); ++k) {
              if (!tet_inside(dd, pp, kuhn, (int)k, kt[k])) continue;
              for (int v = 0; v < 4; ++v) mark_node(level_id(kt[k][v], l));
            }
          };
          if (T.split(d, p)) {
            for (uint64_t cc = 0; cc < 8; ++cc) {
              mark_box(d + 1, (p << 3) | cc);
              add(d + 1, (p << 3) | cc);
            }
          } else {
            mark_box(d, p);
            add(d, p);
          }
          for (int oz = -1; oz <= 1; ++oz)
            for (int oy = -1; oy <= 1; ++oy)
              for (int ox = -1; ox <= 1; ++ox) {
                if (!ox && !oy && !oz) continue;
                int o[3] = {ox, oy, oz};
                uint64_t nq;
                if (!T.offset(d, p, o, nq)) continue;
                int dd = d;
                while (!T.exists(dd, nq)) {
                  --dd;
                  nq >>= 3;
                }
                if (dd == d && T.split(d, nq)) {
                  for (uint64_t cc = 0; cc < 8; ++cc) mark_box(d + 1, (nq << 3) | cc);
                } else {
                  mark_box(dd, nq);
                }
              }
        }
      });
      // gather (contiguous ranges per thread, concatenated in order) and clear
      {
        std::vector<std::vector<int32_t>> sp(nthr);
        pfor((int64_t)AK.size(), [&](unsigned t, int64_t b0, int64_t b1) {
          for (int64_t q = b0; q < b1; ++q)
            if (sflag[q].load(std::memory_order_relaxed)) {
              sp[t].push_back((int32_t)q);
              sflag[q].store(0, std::memory_order_relaxed);
            }
        });
        for (auto& v : sp) L.smooth.insert(L.smooth.end(), v.begin(), v.end());
      }
      for (int dd = 0; dd <= d + 1; ++dd) {
        const auto& bx = BX[dd];
        std::vector<std::vector<std::pair<int, uint64_t>>> rp(nthr);
        pfor((int64_t)bx.size(), [&](unsigned t, int64_t b0, int64_t b1) {
          for (int64_t q = b0; q < b1; ++q)
            if (rflag[dd][q].load(std::memory_order_relaxed)) {
              rp[t].push_back({dd, bx[q]});
              rflag[dd][q].store(0, std::memory_order_relaxed);
            }
        });
        for (auto& v : rp) rel.insert(rel.end(), v.begin(), v.end());
      }
    }
    if (!local) {
      std::sort(rel.begin(), rel.end());
      rel.erase(std::unique(rel.begin(), rel.end()), rel.end());
      uniq(sm);
      for (uint64_t k : sm) L.smooth.push_back(AKI.find(k));
    }
    std::vector<std::vector<int32_t>> ids(nthr);
    std::vector<std::vector<uint64_t>> keys(nthr);
    std::vector<std::vector<double>> coefs(nthr);
    pfor((int64_t)rel.size(), [&](unsigned t, int64_t b0, int64_t b1) {
      std::vector<Tet> kt;  // scratch of this thread
      for (int64_t q = b0; q < b1; ++q) emit_box(rel[q].first, rel[q].second, l, ids[t], keys[t], coefs[t], kt);
    });
    // concatenate in thread order: sizes first, then one copy per part in parallel
    {
      std::vector<size_t> o4(nthr + 1, 0), o1(nthr + 1, 0);
      for (unsigned t = 0; t < nthr; ++t) {
        o4[t + 1] = o4[t] + ids[t].size();
        o1[t + 1] = o1[t] + coefs[t].size();
      }
      L.tri_id.resize(o4[nthr]);
      L.tri_key.resize(o4[nthr]);
      L.tri_coef.resize(o1[nthr]);
      std::vector<std::thread> th;
      for (unsigned t = 0; t < nthr; ++t) {
        if (ids[t].empty() && coefs[t].empty()) continue;
        th.emplace_back([&, t] {
          std::copy(ids[t].begin(), ids[t].end(), L.tri_id.begin() + o4[t]);
          std::copy(keys[t].begin(), keys[t].end(), L.tri_key.begin() + o4[t]);
          std::copy(coefs[t].begin(), coefs[t].end(), L.tri_coef.begin() + o1[t]);
        });
      }
      for (auto& x : th) x.join();
    }
    if (mixed && mesh.nb_layers >= 0) {
      // Algorithm 3: J_{l,j} = the free nodes of the j-th layer of tetrahedra
      // around Gamma_l
      for (uint64_t k : nb::near_boundary_nodes(4, L.tri_key, mesh.nb_layers)) {
        const int32_t id = level_id(k, l);
        if (id >= 0) L.nb_id.push_back(id);
      }
      std::sort(L.nb_id.begin(), L.nb_id.end());
      // A_l[J,J] from the level's kept simplices, factored for the exact
      // near-boundary solve
      std::vector<double> pts(L.tri_key.size() * 3);
      for (size_t k = 0; k < L.tri_key.size(); ++k) lattice_point3(tree, T.LB, L.tri_key[k], &pts[3 * k]);
      nb::assemble_block(3, L.tri_coef.size(), pts.data(), L.tri_coef.data(), L.tri_id.data(), L.nb_id, L.nb_ptr,
                         L.nb_col, L.nb_val);
      if (!nb::factor((int64_t)L.nb_id.size(), L.nb_ptr.data(), L.nb_col.data(), L.nb_val.data(), L.nb_fac))
        ASMG_FAIL(ASMG_ERR_BAD_MESH, "near-boundary block not positive definite");
    }
    if (!dgrid && !mixed) {
      for (auto& v : newnodes[l]) {
        if (bnd3(T, v[0])) continue;
        L.new_id.push_back(AKI.find(v[0]));
        L.new_p0.push_back(bnd3(T, v[1]) ? -1 : AKI.find(v[1]));
        L.new_p1.push_back(bnd3(T, v[2]) ? -1 : AKI.find(v[2]));
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

  // ---- table of the device Scott-Zhang build (Sec. 4.1): the boxes of
  // every depth with their first child or leaf number, the leaves' finest
  // tetrahedra and the aux ID of every vertex (-1 on the boundary)
  {
    SZTable& z = out.sz;
    z.dim = 3;
    z.D = T.LB;
    for (int k = 0; k < 3; ++k) z.amin[k] = tree.amin[k];
    z.L = tree.L;
    std::vector<int64_t> doff(J + 2, 0);
    for (int d = 0; d <= J; ++d) doff[d + 1] = doff[d] + (int64_t)BX[d].size();
    z.node_key.assign(doff[J + 1], 0);
    z.node_pay.assign(doff[J + 1], 0);
    z.leaf_first.assign(nleaf + 1, (int64_t)ftet.size());
    for (int d = 0; d <= J; ++d) {
      const auto& bx = BX[d];
      pfor((int64_t)bx.size(), [&](unsigned, int64_t b0, int64_t b1) {
        for (int64_t i = b0; i < b1; ++i) {
          const int64_t k = doff[d] + i;
          z.node_key[k] = bx[i];
          if (lid[d][i] >= 0) {
            z.node_pay[k] = -((int64_t)lid[d][i] + 1);
            z.leaf_first[lid[d][i]] = first[d][i];
          } else {
            const auto& sd = T.S[d];
            z.node_pay[k] = doff[d + 1] + 8 * (int64_t)(std::lower_bound(sd.begin(), sd.end(), bx[i]) - sd.begin());
          }
        }
      });
    }
    z.simp_key.resize(4 * ftet.size());
    if (!ftet.empty()) std::memcpy(z.simp_key.data(), ftet.data(), ftet.size() * sizeof(ftet[0]));
    z.simp_col.assign(4 * ftet.size(), -1);
    for (int d = 0; d <= J; ++d) {
      const auto& bx = BX[d];
      pfor((int64_t)bx.size(), [&](unsigned, int64_t b0, int64_t b1) {
        for (int64_t i = b0; i < b1; ++i) {
          const int64_t f0 = first[d][i];
          if (f0 < 0) continue;
          const int nq = nft[d][i];
          for (int q = 0; q < nq; ++q) {
            if (!tet_inside(d, bx[i], nq == 6, q, ftet[f0 + q])) continue;  // hats vanish outside Omega^D_J
            for (int v = 0; v < 4; ++v) z.simp_col[4 * (f0 + q) + v] = level_id(ftet[f0 + q][v], J);
          }
        }
      });
    }
  }
}

}  // namespace asmg
