// Exact-overlap primitives of the setup, shared by the host construction
// (auxiliary coefficients) and the device Scott-Zhang kernel:
//   2D  Sutherland-Hodgman clipping of a convex polygon by a triangle, and
//       the polygon moments [1, x, y, x^2, xy, y^2] by Green's theorem;
//   3D  a tetrahedron cut by the four half-spaces of another, visited piece
//       by piece (each plane cut keeps 0, 1 or 3 tetrahedra), and the
//       symmetric 4-point degree-2 rule for products of affine functions.
#pragma once

#include <cmath>
#include <cstdint>

#if defined(__CUDACC__)
#define ASMG_HD __host__ __device__ inline
#else
#define ASMG_HD inline
#endif

namespace asmg {
namespace clip {

// ---------------------------------------------------------------- 2D
struct V2 {
  double x, y;
};

// Clip the convex polygon `in` (CCW) to the half-plane n.x <= c.
ASMG_HD int clip_half(const V2* in, int n, double nx, double ny, double c, V2* out) {
  int m = 0;
  for (int i = 0; i < n; ++i) {
    const V2& a = in[i];
    const V2& b = in[(i + 1) % n];
    const double fa = nx * a.x + ny * a.y - c, fb = nx * b.x + ny * b.y - c;
    if (fa <= 0) out[m++] = a;
    if ((fa <= 0) != (fb <= 0)) {
      const double t = fa / (fa - fb);
      out[m++] = V2{a.x + t * (b.x - a.x), a.y + t * (b.y - a.y)};
    }
  }
  return m;
}

// Clip polygon P (CCW, at most 13 vertices) by triangle K (CCW); out holds 16.
ASMG_HD int clip_tri(const V2* P, int n, const V2* K, V2* out) {
  V2 buf[2][16];
  int m = n;
  for (int i = 0; i < n; ++i) buf[0][i] = P[i];
  int cur = 0;
  for (int e = 0; e < 3 && m >= 3; ++e) {
    const V2& a = K[e];
    const V2& b = K[(e + 1) % 3];
    // inside of a CCW edge a->b: cross(b - a, x - a) >= 0  <=>  n.x <= c
    const double nx = (b.y - a.y), ny = -(b.x - a.x);
    const double c = nx * a.x + ny * a.y;
    m = clip_half(buf[cur], m, nx, ny, c, buf[1 - cur]);
    cur = 1 - cur;
  }
  for (int i = 0; i < m; ++i) out[i] = buf[cur][i];
  return m;
}

// Moments of a polygon by Green's theorem: [1, x, y, x^2, xy, y^2].
ASMG_HD void moments(const V2* p, int n, double M[6]) {
  for (int k = 0; k < 6; ++k) M[k] = 0;
  for (int i = 0; i < n; ++i) {
    const V2& a = p[i];
    const V2& b = p[(i + 1) % n];
    const double c = a.x * b.y - b.x * a.y;
    M[0] += c;
    M[1] += (a.x + b.x) * c;
    M[2] += (a.y + b.y) * c;
    M[3] += (a.x * a.x + a.x * b.x + b.x * b.x) * c;
    M[4] += (a.x * b.y + 2 * a.x * a.y + 2 * b.x * b.y + b.x * a.y) * c;
    M[5] += (a.y * a.y + a.y * b.y + b.y * b.y) * c;
  }
  M[0] /= 2;
  M[1] /= 6;
  M[2] /= 6;
  M[3] /= 12;
  M[4] /= 24;
  M[5] /= 12;
}

// Affine coefficients (c0 + c1 x + c2 y) of the barycentric function of vertex j.
ASMG_HD void bary_affine(const V2* T, int j, double c[3]) {
  const V2 &p = T[(j + 1) % 3], &q = T[(j + 2) % 3];
  const double twoA = (T[1].x - T[0].x) * (T[2].y - T[0].y) - (T[2].x - T[0].x) * (T[1].y - T[0].y);
  c[0] = (p.x * q.y - q.x * p.y) / twoA;
  c[1] = (p.y - q.y) / twoA;
  c[2] = (q.x - p.x) / twoA;
}

// int (f0 + f1 x + f2 y)(g0 + g1 x + g2 y) from the moments
ASMG_HD double prod_int(const double f[3], const double g[3], const double M[6]) {
  return f[0] * g[0] * M[0] + (f[0] * g[1] + f[1] * g[0]) * M[1] + (f[0] * g[2] + f[2] * g[0]) * M[2] +
         f[1] * g[1] * M[3] + (f[1] * g[2] + f[2] * g[1]) * M[4] + f[2] * g[2] * M[5];
}

// ---------------------------------------------------------------- 3D
struct V3 {
  double v[3];
};
struct Tet4 {
  V3 p[4];
};

ASMG_HD double vol6(const V3& a, const V3& b, const V3& c, const V3& d) {
  const double e1[3] = {b.v[0] - a.v[0], b.v[1] - a.v[1], b.v[2] - a.v[2]};
  const double e2[3] = {c.v[0] - a.v[0], c.v[1] - a.v[1], c.v[2] - a.v[2]};
  const double e3[3] = {d.v[0] - a.v[0], d.v[1] - a.v[1], d.v[2] - a.v[2]};
  return e1[0] * (e2[1] * e3[2] - e2[2] * e3[1]) - e1[1] * (e2[0] * e3[2] - e2[2] * e3[0]) +
         e1[2] * (e2[0] * e3[1] - e2[1] * e3[0]);
}

ASMG_HD double volume(const Tet4& t) { return fabs(vol6(t.p[0], t.p[1], t.p[2], t.p[3])) / 6.0; }

ASMG_HD V3 lerp(const V3& a, const V3& b, double da, double db) {
  const double t = da / (da - db);
  return V3{{a.v[0] + t * (b.v[0] - a.v[0]), a.v[1] + t * (b.v[1] - a.v[1]), a.v[2] + t * (b.v[2] - a.v[2])}};
}

// The part of t with n.x - c <= 0 as 0, 1 or 3 tetrahedra (-1: t is kept
// whole).  Vertices are classified by the exact sign of their distance, so
// every intersection parameter lies in [0, 1) and no point moves across the
// plane (pieces of zero volume are harmless).
ASMG_HD int cut_tet(const Tet4& t, const double n[3], double c, Tet4 out[3]) {
  double dv[4];
  int in[4], ni = 0, ou[4], no = 0;
  for (int v = 0; v < 4; ++v) {
    dv[v] = n[0] * t.p[v].v[0] + n[1] * t.p[v].v[1] + n[2] * t.p[v].v[2] - c;
    if (dv[v] <= 0)
      in[ni++] = v;
    else
      ou[no++] = v;
  }
  if (no == 0) return -1;
  if (ni == 0) return 0;
  if (ni == 1) {
    const V3& a = t.p[in[0]];
    out[0] = Tet4{{a, lerp(a, t.p[ou[0]], dv[in[0]], dv[ou[0]]), lerp(a, t.p[ou[1]], dv[in[0]], dv[ou[1]]),
                   lerp(a, t.p[ou[2]], dv[in[0]], dv[ou[2]])}};
    return 1;
  }
  V3 A[3], B[3];
  if (ni == 3) {
    // prism: inside triangle (a0 a1 a2), cut triangle (b0 b1 b2), ak - bk edges
    for (int k = 0; k < 3; ++k) {
      A[k] = t.p[in[k]];
      B[k] = lerp(t.p[in[k]], t.p[ou[0]], dv[in[k]], dv[ou[0]]);
    }
  } else {
    // two inside (i0, i1), two outside (o0, o1): prism with triangles
    // (i0, p00, p01) and (i1, p10, p11)
    const V3 &i0 = t.p[in[0]], &i1 = t.p[in[1]];
    A[0] = i0;
    A[1] = lerp(i0, t.p[ou[0]], dv[in[0]], dv[ou[0]]);
    A[2] = lerp(i0, t.p[ou[1]], dv[in[0]], dv[ou[1]]);
    B[0] = i1;
    B[1] = lerp(i1, t.p[ou[0]], dv[in[1]], dv[ou[0]]);
    B[2] = lerp(i1, t.p[ou[1]], dv[in[1]], dv[ou[1]]);
  }
  out[0] = Tet4{{A[0], A[1], A[2], B[0]}};
  out[1] = Tet4{{A[1], A[2], B[0], B[1]}};
  out[2] = Tet4{{A[2], B[0], B[1], B[2]}};
  return 3;
}

// S cut by the four half-spaces of tetrahedron K: visit(piece) for every
// tetrahedron of S n K, depth first (a piece waits on a stack of at most
// 1 + 2 * 4 entries).  Returns false when the bounding boxes do not overlap
// (no pieces), true otherwise.
template <class F>
ASMG_HD bool clip_tets(const Tet4& S, const Tet4& K, F&& visit) {
  for (int k = 0; k < 3; ++k) {
    double s0 = S.p[0].v[k], s1 = S.p[0].v[k], k0 = K.p[0].v[k], k1 = K.p[0].v[k];
    for (int v = 1; v < 4; ++v) {
      s0 = fmin(s0, S.p[v].v[k]);
      s1 = fmax(s1, S.p[v].v[k]);
      k0 = fmin(k0, K.p[v].v[k]);
      k1 = fmax(k1, K.p[v].v[k]);
    }
    if (s1 <= k0 || k1 <= s0) return false;
  }
  // the four face planes of K, oriented so that K lies on the kept side (the
  // cuts use only signs and ratios of distances: no normalisation needed)
  double pn[4][3], pc[4];
  const int fc[4][4] = {{1, 2, 3, 0}, {0, 2, 3, 1}, {0, 1, 3, 2}, {0, 1, 2, 3}};
  for (int f = 0; f < 4; ++f) {
    const V3 &a = K.p[fc[f][0]], &b = K.p[fc[f][1]], &c = K.p[fc[f][2]], &d = K.p[fc[f][3]];
    const double e1[3] = {b.v[0] - a.v[0], b.v[1] - a.v[1], b.v[2] - a.v[2]};
    const double e2[3] = {c.v[0] - a.v[0], c.v[1] - a.v[1], c.v[2] - a.v[2]};
    double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    double cc = n[0] * a.v[0] + n[1] * a.v[1] + n[2] * a.v[2];
    if (n[0] * d.v[0] + n[1] * d.v[1] + n[2] * d.v[2] > cc) {
      for (int k = 0; k < 3; ++k) n[k] = -n[k];
      cc = -cc;
    }
    for (int k = 0; k < 3; ++k) pn[f][k] = n[k];
    pc[f] = cc;
  }
  Tet4 st[10];
  int lev[10], sp = 0;
  st[sp] = S;
  lev[sp++] = 0;
  while (sp) {
    --sp;
    const Tet4 t = st[sp];
    const int f = lev[sp];
    if (f == 4) {
      visit(t);
      continue;
    }
    Tet4 out[3];
    const int np = cut_tet(t, pn[f], pc[f], out);
    if (np < 0) {
      st[sp] = t;
      lev[sp++] = f + 1;
      continue;
    }
    for (int q = np - 1; q >= 0; --q) {
      st[sp] = out[q];
      lev[sp++] = f + 1;
    }
  }
  return true;
}

// affine function of x: c0 + g.x
struct Aff {
  double c0, g[3];
};

ASMG_HD double aff_at(const Aff& f, const V3& x) { return f.c0 + f.g[0] * x.v[0] + f.g[1] * x.v[1] + f.g[2] * x.v[2]; }

// the barycentric functions of the four vertices of T as affine functions
// (one inverse of the edge matrix)
ASMG_HD void bary_all(const Tet4& T, Aff f[4]) {
  double Jm[3][3];
  for (int k = 1; k <= 3; ++k)
    for (int r = 0; r < 3; ++r) Jm[r][k - 1] = T.p[k].v[r] - T.p[0].v[r];
  const double det = Jm[0][0] * (Jm[1][1] * Jm[2][2] - Jm[1][2] * Jm[2][1]) -
                     Jm[0][1] * (Jm[1][0] * Jm[2][2] - Jm[1][2] * Jm[2][0]) +
                     Jm[0][2] * (Jm[1][0] * Jm[2][1] - Jm[1][1] * Jm[2][0]);
  const double id = 1.0 / det;
  double inv[3][3];
  inv[0][0] = (Jm[1][1] * Jm[2][2] - Jm[1][2] * Jm[2][1]) * id;
  inv[0][1] = (Jm[0][2] * Jm[2][1] - Jm[0][1] * Jm[2][2]) * id;
  inv[0][2] = (Jm[0][1] * Jm[1][2] - Jm[0][2] * Jm[1][1]) * id;
  inv[1][0] = (Jm[1][2] * Jm[2][0] - Jm[1][0] * Jm[2][2]) * id;
  inv[1][1] = (Jm[0][0] * Jm[2][2] - Jm[0][2] * Jm[2][0]) * id;
  inv[1][2] = (Jm[0][2] * Jm[1][0] - Jm[0][0] * Jm[1][2]) * id;
  inv[2][0] = (Jm[1][0] * Jm[2][1] - Jm[1][1] * Jm[2][0]) * id;
  inv[2][1] = (Jm[0][1] * Jm[2][0] - Jm[0][0] * Jm[2][1]) * id;
  inv[2][2] = (Jm[0][0] * Jm[1][1] - Jm[0][1] * Jm[1][0]) * id;
  for (int j = 0; j < 4; ++j) {
    for (int r = 0; r < 3; ++r) f[j].g[r] = j == 0 ? -(inv[0][r] + inv[1][r] + inv[2][r]) : inv[j - 1][r];
    f[j].c0 = 1.0 * (j == 0) - (f[j].g[0] * T.p[0].v[0] + f[j].g[1] * T.p[0].v[1] + f[j].g[2] * T.p[0].v[2]);
  }
}

// acc[w] += int over tetrahedron t of f * g[w] for every w with use[w], by
// the symmetric 4-point degree-2 rule: points a v_i + b (sum of the other
// three vertices) with a = (5 + 3 sqrt 5)/20, b = (5 - sqrt 5)/20, weights
// |t|/4.
ASMG_HD void prod4(const Tet4& t, const Aff& f, const Aff* g, const bool* use, double* acc) {
  const double r5 = 2.23606797749978969641;  // sqrt 5
  const double a = (5.0 + 3.0 * r5) / 20.0, b = (5.0 - r5) / 20.0;
  const double w = volume(t) / 4.0;
  for (int i = 0; i < 4; ++i) {
    V3 x;
    for (int k = 0; k < 3; ++k)
      x.v[k] = a * t.p[i].v[k] + b * (t.p[(i + 1) % 4].v[k] + t.p[(i + 2) % 4].v[k] + t.p[(i + 3) % 4].v[k]);
    const double fx = aff_at(f, x) * w;
    for (int j = 0; j < 4; ++j)
      if (use[j]) acc[j] += fx * aff_at(g[j], x);
  }
}

}  // namespace clip
}  // namespace asmg
