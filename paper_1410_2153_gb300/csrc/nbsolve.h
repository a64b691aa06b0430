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

}  // namespace nb
}  // namespace asmg
