// One row of the Scott-Zhang transfer (Sec. 4.1), shared by the device
// kernels of transfer.cu: for the free fine vertex i, P_ik = int_{sigma_i}
// psi_i phi^J_k with sigma_i the lowest-index element at i and psi_i its dual
// basis function (2D: (12 lambda_i - 3)/|sigma_i|, 3D: (20 lambda_i -
// 4)/|sigma_i|).  The row walks the closed tree (SZTable's node table) to the
// leaves whose boxes meet sigma_i's lattice window and clips sigma_i against
// their finest simplices exactly (clip.h).
#pragma once

#include <cstdint>

#include "clip.h"

namespace asmg {
namespace szrow {

using namespace clip;

struct SZDev {
  int dim, D;
  double amin[3], L, sc;  // sc = 2^D / L: lattice units per length
  const uint64_t* node_key;
  const int64_t* node_pay;
  const int64_t* leaf_first;
  const uint64_t* simp_key;
  const int32_t* simp_col;
  const double* X;
  const int32_t* E;
  const int32_t* sigma;
  const int32_t* vof;
  int64_t n;
  int64_t nnode, nleaf, nsimp, nv, ne;  // array sizes: every index is checked against them
};

constexpr int STACK = 32;  // tree depth limit of the traversal

ASMG_HD uint64_t compact2(uint64_t v) {
  v &= 0x5555555555555555ULL;
  v = (v | (v >> 1)) & 0x3333333333333333ULL;
  v = (v | (v >> 2)) & 0x0F0F0F0F0F0F0F0FULL;
  v = (v | (v >> 4)) & 0x00FF00FF00FF00FFULL;
  v = (v | (v >> 8)) & 0x0000FFFF0000FFFFULL;
  v = (v | (v >> 16)) & 0x00000000FFFFFFFFULL;
  return v;
}

ASMG_HD uint64_t compact3(uint64_t v) {
  v &= 0x1249249249249249ULL;
  v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ULL;
  v = (v ^ (v >> 4)) & 0x100f00f00f00f00fULL;
  v = (v ^ (v >> 8)) & 0x1f0000ff0000ffULL;
  v = (v ^ (v >> 16)) & 0x1f00000000ffffULL;
  v = (v ^ (v >> 32)) & 0x1fffffULL;
  return v;
}

ASMG_HD void key_xyz(const SZDev& t, uint64_t key, uint64_t* q) {
  if (t.dim == 2) {
    q[0] = compact2(key);
    q[1] = compact2(key >> 1);
    q[2] = 0;
  } else {
    q[0] = compact3(key);
    q[1] = compact3(key >> 1);
    q[2] = compact3(key >> 2);
  }
}

// f(leaf) for every leaf whose box meets the lattice window [lo, hi]: in 2D
// closed boxes against the closed window, in 3D with positive overlap.
// Depth first, one stack entry per depth: the first child of the box being
// expanded and the next child to visit.  Returns false if the tree is deeper
// than the stack or an index leaves its array (the caller flags an error).
template <class F>
ASMG_HD bool for_leaves(const SZDev& t, const int64_t* lo, const int64_t* hi, F&& f) {
  const int nch = t.dim == 2 ? 4 : 8;
  int64_t base[STACK];
  int next[STACK];
  int top = -1;
  int64_t k = 0;  // the node to visit and its depth
  int d = 0;
  for (;;) {
    if (k < 0 || k >= t.nnode) return false;
    const int64_t s = 1LL << (t.D - d);
    uint64_t q[3];
    key_xyz(t, t.node_key[k], q);
    bool meet = true;
    for (int a = 0; a < t.dim; ++a) {
      const int64_t x0 = (int64_t)q[a] * s;
      if (t.dim == 2 ? (x0 > hi[a] || x0 + s < lo[a]) : (x0 >= hi[a] || x0 + s <= lo[a])) meet = false;
    }
    if (meet) {
      const int64_t pay = t.node_pay[k];
      if (pay < 0) {
        const int64_t leaf = -pay - 1;
        if (leaf >= t.nleaf || t.leaf_first[leaf] < 0 || t.leaf_first[leaf + 1] > t.nsimp) return false;
        f(leaf);
      } else {
        if (top + 1 >= STACK) return false;
        ++top;
        base[top] = pay;
        next[top] = 0;
      }
    }
    while (top >= 0 && next[top] == nch) --top;
    if (top < 0) return true;
    k = base[top] + next[top];
    next[top] += 1;
    d = top + 1;
  }
}

ASMG_HD double lat(const SZDev& t, uint64_t q, int a) {
  return t.amin[a] + ldexp((double)q, -t.D) * t.L;
}

// One row: emit(col, value) for every (simplex, free vertex) contribution
// (values computed only when `values` is set; 0 is passed otherwise).
// Returns false when an index leaves its array.
template <int DIM, class Emit>
ASMG_HD bool sz_row(const SZDev& t, int64_t i, bool values, Emit&& emit) {
  const int32_t v = t.vof[i];
  if (v < 0 || v >= t.nv) return false;
  const int64_t e = t.sigma[v];
  if (e < 0 || e >= t.ne) return false;
  for (int k = 0; k <= DIM; ++k)
    if (t.E[(DIM + 1) * e + k] < 0 || t.E[(DIM + 1) * e + k] >= t.nv) return false;
  if (DIM == 2) {
    V2 P[3];
    int loc = 0;
    for (int k = 0; k < 3; ++k) {
      const int32_t w = t.E[3 * e + k];
      P[k] = V2{t.X[2 * (int64_t)w], t.X[2 * (int64_t)w + 1]};
      if (w == v) loc = k;
    }
    const V2 o = P[0];
    V2 Pl[3];
    for (int k = 0; k < 3; ++k) Pl[k] = V2{P[k].x - o.x, P[k].y - o.y};
    const double area = 0.5 * (Pl[1].x * Pl[2].y - Pl[2].x * Pl[1].y);
    double lam[3], psi[3];
    bary_affine(Pl, loc, lam);
    psi[0] = (12.0 * lam[0] - 3.0) / area;
    psi[1] = 12.0 * lam[1] / area;
    psi[2] = 12.0 * lam[2] / area;
    const double mnx = fmin(fmin(P[0].x, P[1].x), P[2].x), mxx = fmax(fmax(P[0].x, P[1].x), P[2].x);
    const double mny = fmin(fmin(P[0].y, P[1].y), P[2].y), mxy = fmax(fmax(P[0].y, P[1].y), P[2].y);
    const int64_t lo[2] = {(int64_t)floor((mnx - t.amin[0]) * t.sc) - 2, (int64_t)floor((mny - t.amin[1]) * t.sc) - 2};
    const int64_t hi[2] = {(int64_t)ceil((mxx - t.amin[0]) * t.sc) + 2, (int64_t)ceil((mxy - t.amin[1]) * t.sc) + 2};
    return for_leaves(t, lo, hi, [&](int64_t leaf) {
      for (int64_t q = t.leaf_first[leaf]; q < t.leaf_first[leaf + 1]; ++q) {
        V2 K[3];
        for (int k = 0; k < 3; ++k) {
          uint64_t c[3];
          key_xyz(t, t.simp_key[3 * q + k], c);
          K[k] = V2{lat(t, c[0], 0) - o.x, lat(t, c[1], 1) - o.y};
        }
        V2 poly[16];
        const int m = clip_tri(Pl, 3, K, poly);
        if (m < 3) continue;
        double M[6];
        moments(poly, m, M);
        if (!(M[0] > 0)) continue;
        for (int k = 0; k < 3; ++k) {
          const int32_t col = t.simp_col[3 * q + k];
          if (col < 0) continue;
          double val = 0;
          if (values) {
            double phi[3];
            bary_affine(K, k, phi);
            val = prod_int(psi, phi, M);
          }
          emit(col, val);
        }
      }
    });
  }
  Tet4 S;
  int loc = 0;
  for (int k = 0; k < 4; ++k) {
    const int32_t w = t.E[4 * e + k];
    for (int a = 0; a < 3; ++a) S.p[k].v[a] = t.X[3 * (int64_t)w + a];
    if (w == v) loc = k;
  }
  int64_t lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    double mn = S.p[0].v[a], mx = S.p[0].v[a];
    for (int k = 1; k < 4; ++k) {
      mn = fmin(mn, S.p[k].v[a]);
      mx = fmax(mx, S.p[k].v[a]);
    }
    // widened by 1e-9 lattice units against rounding of the scaling
    lo[a] = (int64_t)floor((mn - t.amin[a]) * t.sc - 1e-9);
    hi[a] = (int64_t)ceil((mx - t.amin[a]) * t.sc + 1e-9);
  }
  Aff psi;
  {
    const double vol = volume(S);
    Aff lam[4];
    bary_all(S, lam);
    psi.c0 = (20.0 * lam[loc].c0 - 4.0) / vol;
    for (int a = 0; a < 3; ++a) psi.g[a] = 20.0 * lam[loc].g[a] / vol;
  }
  return for_leaves(t, lo, hi, [&](int64_t leaf) {
    for (int64_t q = t.leaf_first[leaf]; q < t.leaf_first[leaf + 1]; ++q) {
      int32_t col[4];
      bool use[4], any = false;
      for (int w = 0; w < 4; ++w) {
        col[w] = t.simp_col[4 * q + w];
        use[w] = col[w] >= 0;
        any = any || use[w];
      }
      if (!any) continue;
      Tet4 K;
      for (int k = 0; k < 4; ++k) {
        uint64_t c[3];
        key_xyz(t, t.simp_key[4 * q + k], c);
        for (int a = 0; a < 3; ++a) K.p[k].v[a] = lat(t, c[a], a);
      }
      Aff phi[4];
      if (values) bary_all(K, phi);
      double val[4] = {0, 0, 0, 0};
      int npiece = 0;
      clip_tets(S, K, [&](const Tet4& pc) {
        ++npiece;
        if (values) prod4(pc, psi, phi, use, val);
      });
      if (!npiece) continue;
      for (int w = 0; w < 4; ++w)
        if (use[w]) emit(col[w], val[w]);
    }
  });
}

// Pass `mode` of the row pipeline for row i: 0 counts the contributions into
// cnt[i]; 1 writes them into [off[i], off[i + 1]) and stores how many it
// wrote in cnt[i] (false if that differs from the slot).  Both passes take
// the same decisions (the values do not steer them), so they see the same
// contributions.
template <int DIM>
ASMG_HD bool sz_pass(const SZDev& t, int64_t i, int mode, const int64_t* off, int64_t* cnt, int32_t* col,
                     double* val, bool* stack_ok) {
  int64_t c = 0;
  const int64_t b = mode ? off[i] : 0, e = mode ? off[i + 1] : 0;
  *stack_ok = sz_row<DIM>(t, i, mode != 0, [&](int32_t k, double v) {
    if (mode && b + c < e) {
      col[b + c] = k;
      val[b + c] = v;
    }
    ++c;
  });
  cnt[i] = mode ? (c < e - b ? c : e - b) : c;
  return !mode || c == e - b;
}

// Sort row i's slot by column (insertion sort, stable: duplicates are added
// in traversal order), add duplicates in place; returns the merged length.
ASMG_HD int64_t sz_merge(int64_t i, const int64_t* off, const int64_t* cnt, int32_t* col, double* val) {
  const int64_t b = off[i], e = b + cnt[i];
  for (int64_t p = b + 1; p < e; ++p) {
    const int32_t c = col[p];
    const double v = val[p];
    int64_t q = p - 1;
    while (q >= b && col[q] > c) {
      col[q + 1] = col[q];
      val[q + 1] = val[q];
      --q;
    }
    col[q + 1] = c;
    val[q + 1] = v;
  }
  int64_t m = b;
  for (int64_t p = b; p < e;) {
    int64_t q = p;
    double s = 0;
    while (q < e && col[q] == col[p]) s += val[q++];
    col[m] = col[p];
    val[m] = s;
    ++m;
    p = q;
  }
  return m - b;
}

}  // namespace szrow
}  // namespace asmg
