// Exact solve on the near-boundary set J_{l,j} of Algorithm 3: x = (A_JJ)^{-1} b
// for the symmetric positive definite block A_JJ of a level operator.
//
// The nodes of J_{l,j} form a strip a few elements wide along the boundary
// curves (surfaces) of the level.  Ordered by breadth-first level sets (from a
// node of least degree, per connected component), A_JJ is block tridiagonal:
// an edge joins nodes of the same or of neighbouring level sets only.  Block
// cyclic reduction eliminates the odd blocks of each round in parallel and
// leaves a block-tridiagonal system on the even ones, so a solve takes
// 2 ceil(log2(#blocks)) rounds whose blocks are independent: the form a device
// kernel applies, one thread block per block.  The factorisation is done once
// at setup, in FP64 on the host.
#pragma once

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <vector>

namespace asmg {
namespace nb {

// dense row-major blocks
struct Blk {
  int r = 0, c = 0;
  std::vector<double> a;
  Blk() = default;
  Blk(int r_, int c_) : r(r_), c(c_), a((size_t)r_ * c_, 0.0) {}
  double& at(int i, int j) { return a[(size_t)i * c + j]; }
  double at(int i, int j) const { return a[(size_t)i * c + j]; }
  bool empty() const { return r == 0 || c == 0; }
};

// C -= A * B
inline void gemm_sub(const Blk& A, const Blk& B, Blk& C) {
  for (int i = 0; i < A.r; ++i)
    for (int k = 0; k < A.c; ++k) {
      const double v = A.at(i, k);
      if (v == 0) continue;
      for (int j = 0; j < B.c; ++j) C.at(i, j) -= v * B.at(k, j);
    }
}

// lower Cholesky factor in place; false if not positive definite
inline bool chol(Blk& D) {
  for (int j = 0; j < D.r; ++j) {
    double s = D.at(j, j);
    for (int k = 0; k < j; ++k) s -= D.at(j, k) * D.at(j, k);
    if (!(s > 0)) return false;
    D.at(j, j) = std::sqrt(s);
    for (int i = j + 1; i < D.r; ++i) {
      double t = D.at(i, j);
      for (int k = 0; k < j; ++k) t -= D.at(i, k) * D.at(j, k);
      D.at(i, j) = t / D.at(j, j);
    }
    for (int k = j + 1; k < D.r; ++k) D.at(j, k) = 0;
  }
  return true;
}

// X := D^{-1} X for the Cholesky factor stored in F (every column of X)
inline void chol_solve(const Blk& F, Blk& X) {
  for (int col = 0; col < X.c; ++col) {
    for (int i = 0; i < F.r; ++i) {
      double s = X.at(i, col);
      for (int k = 0; k < i; ++k) s -= F.at(i, k) * X.at(k, col);
      X.at(i, col) = s / F.at(i, i);
    }
    for (int i = F.r - 1; i >= 0; --i) {
      double s = X.at(i, col);
      for (int k = i + 1; k < F.r; ++k) s -= F.at(k, i) * X.at(k, col);
      X.at(i, col) = s / F.at(i, i);
    }
  }
}

// One round of the reduction: blocks 0..n-1 of the current system with their
// diagonal D[k], coupling Lo[k] to block k-1 and Up[k] to block k+1.
struct Round {
  std::vector<Blk> F;       // Cholesky factors of the odd blocks' D
  std::vector<Blk> Lo, Up;  // couplings of every block of this round
  int n = 0;
};

struct Factor {
  int64_t m = 0;
  std::vector<int32_t> order;   // ordered position -> row of A_JJ
  std::vector<int64_t> bstart;  // block b holds ordered positions [bstart[b], bstart[b + 1])
  std::vector<Round> rounds;
  Blk last;                     // Cholesky factor of the single block left
  bool ok = false;
};

// Breadth-first level sets of the graph of A (CSR, symmetric pattern), each
// component from a node of least degree; components one after another.
inline void level_sets(int64_t m, const int64_t* ptr, const int32_t* col, std::vector<int32_t>& order,
                       std::vector<int64_t>& bstart) {
  std::vector<int32_t> lev(m, -1);
  order.clear();
  bstart.assign(1, 0);
  std::vector<int32_t> byDeg(m);
  for (int64_t i = 0; i < m; ++i) byDeg[i] = (int32_t)i;
  std::stable_sort(byDeg.begin(), byDeg.end(),
                   [&](int32_t a, int32_t b) { return ptr[a + 1] - ptr[a] < ptr[b + 1] - ptr[b]; });
  for (int32_t s : byDeg) {
    if (lev[s] >= 0) continue;
    std::vector<int32_t> cur(1, s), next;
    lev[s] = 0;
    while (!cur.empty()) {
      std::sort(cur.begin(), cur.end());
      order.insert(order.end(), cur.begin(), cur.end());
      bstart.push_back((int64_t)order.size());
      next.clear();
      for (int32_t v : cur)
        for (int64_t p = ptr[v]; p < ptr[v + 1]; ++p)
          if (col[p] != v && lev[col[p]] < 0) {
            lev[col[p]] = 1;
            next.push_back(col[p]);
          }
      cur.swap(next);
    }
  }
}

// Factor A_JJ (CSR, m rows, symmetric positive definite).
inline bool factor(int64_t m, const int64_t* ptr, const int32_t* col, const double* val, Factor& Fz) {
  Fz = Factor();
  Fz.m = m;
  Fz.ok = true;
  if (m == 0) return true;
  level_sets(m, ptr, col, Fz.order, Fz.bstart);
  const int nb = (int)Fz.bstart.size() - 1;
  std::vector<int32_t> pos(m), blk(m);
  for (int64_t q = 0; q < m; ++q) pos[Fz.order[q]] = (int32_t)q;
  for (int b = 0; b < nb; ++b)
    for (int64_t q = Fz.bstart[b]; q < Fz.bstart[b + 1]; ++q) blk[Fz.order[q]] = b;
  std::vector<Blk> D(nb), Lo(nb), Up(nb);
  for (int b = 0; b < nb; ++b) {
    const int nbk = (int)(Fz.bstart[b + 1] - Fz.bstart[b]);
    D[b] = Blk(nbk, nbk);
    if (b > 0) Lo[b] = Blk(nbk, (int)(Fz.bstart[b] - Fz.bstart[b - 1]));
    if (b + 1 < nb) Up[b] = Blk(nbk, (int)(Fz.bstart[b + 2] - Fz.bstart[b + 1]));
  }
  for (int64_t i = 0; i < m; ++i) {
    const int bi = blk[i];
    const int li = (int)(pos[i] - Fz.bstart[bi]);
    for (int64_t p = ptr[i]; p < ptr[i + 1]; ++p) {
      const int32_t j = col[p];
      const int bj = blk[j];
      const int lj = (int)(pos[j] - Fz.bstart[bj]);
      if (bj == bi) D[bi].at(li, lj) += val[p];
      else if (bj == bi - 1) Lo[bi].at(li, lj) += val[p];
      else if (bj == bi + 1) Up[bi].at(li, lj) += val[p];
      else return Fz.ok = false;  // not block tridiagonal (cannot happen for level sets)
    }
  }
  // rounds: eliminate the odd blocks; the even ones form the next system
  while ((int)D.size() > 1) {
    const int n = (int)D.size();
    Round R;
    R.n = n;
    R.Lo = Lo;
    R.Up = Up;
    R.F.assign(n, Blk());
    std::vector<Blk> WL(n), WU(n);  // D^{-1} Lo, D^{-1} Up of the odd blocks
    for (int k = 1; k < n; k += 2) {
      R.F[k] = D[k];
      if (!chol(R.F[k])) return Fz.ok = false;
      WL[k] = Lo[k];
      chol_solve(R.F[k], WL[k]);
      if (k + 1 < n) {
        WU[k] = Up[k];
        chol_solve(R.F[k], WU[k]);
      }
    }
    const int ne = (n + 1) / 2;
    std::vector<Blk> D2(ne), L2(ne), U2(ne);
    for (int e = 0; e < n; e += 2) {
      const int h = e / 2;
      D2[h] = D[e];
      if (e - 1 >= 0) {  // previous odd block p = e - 1
        gemm_sub(Lo[e], WU[e - 1], D2[h]);
        if (e - 2 >= 0) {
          L2[h] = Blk(D[e].r, D[e - 2].r);
          gemm_sub(Lo[e], WL[e - 1], L2[h]);
        }
      }
      if (e + 1 < n) {  // next odd block q = e + 1
        gemm_sub(Up[e], WL[e + 1], D2[h]);
        if (e + 2 < n) {
          U2[h] = Blk(D[e].r, D[e + 2].r);
          gemm_sub(Up[e], WU[e + 1], U2[h]);
        }
      }
    }
    Fz.rounds.push_back(std::move(R));
    D.swap(D2);
    Lo.swap(L2);
    Up.swap(U2);
  }
  Fz.last = D[0];
  if (!chol(Fz.last)) return Fz.ok = false;
  return true;
}

// x = A_JJ^{-1} b (b and x indexed like the rows of A_JJ)
inline void solve(const Factor& Fz, const double* b, double* x) {
  if (Fz.m == 0) return;
  const int nb = (int)Fz.bstart.size() - 1;
  std::vector<Blk> rhs(nb);
  for (int k = 0; k < nb; ++k) {
    rhs[k] = Blk((int)(Fz.bstart[k + 1] - Fz.bstart[k]), 1);
    for (int64_t q = Fz.bstart[k]; q < Fz.bstart[k + 1]; ++q) rhs[k].at((int)(q - Fz.bstart[k]), 0) = b[Fz.order[q]];
  }
  // forward: per round, y_odd = D^{-1} b_odd, then b_even -= Lo y_prev + Up y_next
  std::vector<std::vector<Blk>> keep;  // the right-hand sides of each round
  for (const Round& R : Fz.rounds) {
    keep.push_back(rhs);
    std::vector<Blk> y(R.n);
    for (int k = 1; k < R.n; k += 2) {
      y[k] = rhs[k];
      chol_solve(R.F[k], y[k]);
    }
    std::vector<Blk> nx((R.n + 1) / 2);
    for (int e = 0; e < R.n; e += 2) {
      nx[e / 2] = rhs[e];
      if (e - 1 >= 0) gemm_sub(R.Lo[e], y[e - 1], nx[e / 2]);
      if (e + 1 < R.n) gemm_sub(R.Up[e], y[e + 1], nx[e / 2]);
    }
    rhs.swap(nx);
  }
  std::vector<Blk> sol(1, rhs[0]);
  chol_solve(Fz.last, sol[0]);
  // backward: x_odd = D^{-1} (b_odd - Lo x_prev - Up x_next) with the round's b
  for (int r = (int)Fz.rounds.size() - 1; r >= 0; --r) {
    const Round& R = Fz.rounds[r];
    const std::vector<Blk>& br = keep[r];
    std::vector<Blk> full(R.n);
    for (int e = 0; e < R.n; e += 2) full[e] = sol[e / 2];
    for (int k = 1; k < R.n; k += 2) {
      full[k] = br[k];
      gemm_sub(R.Lo[k], full[k - 1], full[k]);
      if (k + 1 < R.n) gemm_sub(R.Up[k], full[k + 1], full[k]);
      chol_solve(R.F[k], full[k]);
    }
    sol.swap(full);
  }
  for (int k = 0; k < nb; ++k)
    for (int64_t q = Fz.bstart[k]; q < Fz.bstart[k + 1]; ++q) x[Fz.order[q]] = sol[k].at((int)(q - Fz.bstart[k]), 0);
}

// The nodes of the near-boundary region T_(l,j) of Algorithm 3 for the kept
// simplices of a level (nv = dim + 1 lattice keys each, in `keys`): layer 0
// is the simplices touching the boundary of their union (the vertices of the
// facets that belong to one simplex only), layer i those touching layer
// i - 1.  On a conforming grid these are the nodes within j + 1 edges of a
// boundary vertex: a breadth-first search over the simplices' edges.
// Returns the node keys, ascending.
inline std::vector<uint64_t> near_boundary_nodes(int nv, const std::vector<uint64_t>& keys, int layers) {
  std::vector<uint64_t> nodes(keys);
  std::sort(nodes.begin(), nodes.end());
  nodes.erase(std::unique(nodes.begin(), nodes.end()), nodes.end());
  auto loc = [&](uint64_t k) { return (int64_t)(std::lower_bound(nodes.begin(), nodes.end(), k) - nodes.begin()); };
  const size_t ns = keys.size() / nv;
  std::vector<std::array<int64_t, 3>> facets;  // sorted vertex positions (third -1 in 2D)
  std::vector<std::array<int64_t, 2>> edges;
  for (size_t t = 0; t < ns; ++t) {
    int64_t v[4];
    for (int k = 0; k < nv; ++k) v[k] = loc(keys[nv * t + k]);
    for (int k = 0; k < nv; ++k) {
      std::array<int64_t, 3> f = {-1, -1, -1};
      int q = 0;
      for (int w = 0; w < nv; ++w)
        if (w != k) f[q++] = v[w];
      std::sort(f.begin(), f.begin() + q);
      facets.push_back(f);
      for (int k2 = k + 1; k2 < nv; ++k2) edges.push_back({std::min(v[k], v[k2]), std::max(v[k], v[k2])});
    }
  }
  std::sort(facets.begin(), facets.end());
  std::sort(edges.begin(), edges.end());
  edges.erase(std::unique(edges.begin(), edges.end()), edges.end());
  std::vector<int32_t> dist(nodes.size(), -1);
  std::vector<int64_t> frontier;
  for (size_t i = 0; i < facets.size();) {
    size_t j = i;
    while (j < facets.size() && facets[j] == facets[i]) ++j;
    if (j - i == 1)
      for (int k = 0; k < nv - 1; ++k)
        if (dist[facets[i][k]] < 0) {
          dist[facets[i][k]] = 0;
          frontier.push_back(facets[i][k]);
        }
    i = j;
  }
  std::vector<int64_t> adjs(nodes.size() + 1, 0), adj(2 * edges.size());
  for (auto& e : edges) {
    adjs[e[0] + 1] += 1;
    adjs[e[1] + 1] += 1;
  }
  for (size_t i = 0; i < nodes.size(); ++i) adjs[i + 1] += adjs[i];
  {
    std::vector<int64_t> fill(adjs.begin(), adjs.end() - 1);
    for (auto& e : edges) {
      adj[fill[e[0]]++] = e[1];
      adj[fill[e[1]]++] = e[0];
    }
  }
  for (int r = 1; r <= layers + 1 && !frontier.empty(); ++r) {
    std::vector<int64_t> next;
    for (int64_t v : frontier)
      for (int64_t q = adjs[v]; q < adjs[v + 1]; ++q)
        if (dist[adj[q]] < 0) {
          dist[adj[q]] = r;
          next.push_back(adj[q]);
        }
    frontier.swap(next);
  }
  std::vector<uint64_t> out;
  for (size_t i = 0; i < nodes.size(); ++i)
    if (dist[i] >= 0) out.push_back(nodes[i]);
  return out;
}

// The block A_l[J,J] of a level operator from the level's simplices: pts
// holds the (dim + 1) vertices of each simplex (dim coordinates each), ids
// their aux IDs (-1: Dirichlet), coef the simplex coefficients; J = nb_id
// (ascending aux IDs).  Entry (p, q) of the block is the sum over the
// simplices holding nb_id[p] and nb_id[q] of coef |tau| grad lambda_p .
// grad lambda_q (P1 stiffness); CSR with ascending columns.
inline void assemble_block(int dim, size_t nsimp, const double* pts, const double* coef, const int32_t* ids,
                           const std::vector<int32_t>& nb_id, std::vector<int64_t>& ptr, std::vector<int32_t>& col,
                           std::vector<double>& val) {
  const int nv = dim + 1;
  std::vector<std::vector<std::pair<int32_t, double>>> rows(nb_id.size());
  for (size_t t = 0; t < nsimp; ++t) {
    int32_t loc[4];
    int nin = 0;
    for (int v = 0; v < nv; ++v) {
      const int32_t id = ids[nv * t + v];
      auto it = std::lower_bound(nb_id.begin(), nb_id.end(), id);
      loc[v] = (id >= 0 && it != nb_id.end() && *it == id) ? (int32_t)(it - nb_id.begin()) : -1;
      nin += loc[v] >= 0;
    }
    if (!nin) continue;
    const double* P = pts + (size_t)nv * dim * t;
    double M[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, inv[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int k = 1; k <= dim; ++k)
      for (int r = 0; r < dim; ++r) M[r][k - 1] = P[k * dim + r] - P[r];
    double det;
    if (dim == 2) {
      det = M[0][0] * M[1][1] - M[0][1] * M[1][0];
      inv[0][0] = M[1][1] / det;
      inv[0][1] = -M[0][1] / det;
      inv[1][0] = -M[1][0] / det;
      inv[1][1] = M[0][0] / det;
    } else {
      det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
            M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
      inv[0][0] = (M[1][1] * M[2][2] - M[1][2] * M[2][1]) / det;
      inv[0][1] = (M[0][2] * M[2][1] - M[0][1] * M[2][2]) / det;
      inv[0][2] = (M[0][1] * M[1][2] - M[0][2] * M[1][1]) / det;
      inv[1][0] = (M[1][2] * M[2][0] - M[1][0] * M[2][2]) / det;
      inv[1][1] = (M[0][0] * M[2][2] - M[0][2] * M[2][0]) / det;
      inv[1][2] = (M[0][2] * M[1][0] - M[0][0] * M[1][2]) / det;
      inv[2][0] = (M[1][0] * M[2][1] - M[1][1] * M[2][0]) / det;
      inv[2][1] = (M[0][1] * M[2][0] - M[0][0] * M[2][1]) / det;
      inv[2][2] = (M[0][0] * M[1][1] - M[0][1] * M[1][0]) / det;
    }
    // row k-1 of M^{-1} is grad lambda_k (k >= 1); grad lambda_0 = -sum
    double G[4][3];
    for (int r = 0; r < dim; ++r) {
      G[0][r] = 0;
      for (int k = 1; k <= dim; ++k) {
        G[k][r] = inv[k - 1][r];
        G[0][r] -= inv[k - 1][r];
      }
    }
    const double vol = std::fabs(det) / (dim == 2 ? 2.0 : 6.0);
    for (int i = 0; i < nv; ++i) {
      if (loc[i] < 0) continue;
      for (int j = 0; j < nv; ++j) {
        if (loc[j] < 0) continue;
        double g = 0;
        for (int r = 0; r < dim; ++r) g += G[i][r] * G[j][r];
        rows[loc[i]].push_back({loc[j], coef[t] * vol * g});
      }
    }
  }
  ptr.assign(nb_id.size() + 1, 0);
  col.clear();
  val.clear();
  for (size_t i = 0; i < rows.size(); ++i) {
    auto& r = rows[i];
    std::stable_sort(r.begin(), r.end(),
                     [](const std::pair<int32_t, double>& a, const std::pair<int32_t, double>& b) { return a.first < b.first; });
    for (size_t k = 0; k < r.size();) {
      size_t j = k;
      double sum = 0;
      while (j < r.size() && r[j].first == r[k].first) sum += r[j++].second;
      col.push_back(r[k].first);
      val.push_back(sum);
      k = j;
    }
    ptr[i + 1] = (int64_t)col.size();
  }
}

}  // namespace nb
}  // namespace asmg
